"""Element-wise parity of the surrogate's kernels, layer by layer.

After one training step on windows of the CPU oracle, the library hands back every intermediate
array of that step (rod_surrogate_debug_buffer): the BF16 activations, the FP32
pre-activations, the output, the loss gradient and the back-propagated BF16 gradients.  Each
layer is then checked on its own, against an FP64 evaluation of the same layer from the GPU's
own inputs to that layer, so no rounding decision taken earlier can blur the comparison:

  * pre-activations and outputs: |z_gpu - z| <= (K + 2) 2^-22 (sum |W a| + |b|) for every entry,
    K = 5 C_in products of BF16 operands (exact in FP32) accumulated in FP32 by the tensor cores
    (2^-22: two units of FP32 rounding per addition, for accumulators that truncate);
  * activations and gradients stored in BF16: the stored value lies in the BF16 rounding of the
    interval that the FP32 value can occupy (the bound above, widened by the error of the FP32
    SiLU or SiLU' evaluation: (5 + 1.2 |x|) 2^-23 relative for the exponential and quotient
    intrinsics, and 1.5e-36 absolute below x = -87, where the fast quotient returns -0);
  * loss gradient: 2 (out - tgt) / count with four FP32 roundings, rounded to BF16;
  * loss: (n + 4) 2^-23 of the sum of the n squared residuals (FP32 sums in any order);
  * weight and bias gradients: (M + 4) 2^-22 (sum |g a|) for M = windows x 64 positions of a chunk.

A dropped, repeated or misplaced tap or channel moves an entry by about one term of its sum,
|W a| ~ (sum |W a|) / K, two orders of magnitude above these bounds.
"""
import numpy as np
import pytest

import rodgen
from oracle import surrogate_ref as R
from test_gpu_surrogate import _act, _cuda, _setup_network, oracle_window  # noqa: F401

pytestmark = pytest.mark.gpu

U22 = 2.0 ** -22
U23 = 2.0 ** -23


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _cp(buf):
    """[windows, rows, channels] with rows = positions + 2 -> [windows, channels, 51]."""
    return np.asarray(buf, dtype=np.float64)[:, 2:2 + R.POS, :].transpose(0, 2, 1)


def _silu_rel(pre):
    """Relative error bound of the FP32 SiLU x / (1 + exp(-x)) with the fast exponential
    (2 + 1.173 |x| units in the last place) and the fast quotient (2 units)."""
    return (5.0 + 1.2 * np.abs(pre)) * U23


def _silu_abs(pre):
    """Absolute slack of the same SiLU: below x = -87.3 the denominator passes 2^126 (or the
    exponential overflows FP32) and the fast quotient returns -0; the true value, |x| e^x, is
    below 1.5e-36 there."""
    return np.where(pre < -87.0, 1.5e-36, 1e-38)


def _bf16_bracket(got, lo, hi):
    """True where the BF16 value `got` is a round-to-nearest BF16 of some value in [lo, hi]."""
    a, b = np.minimum(lo, hi), np.maximum(lo, hi)
    return (R.bf16(a) <= got) & (got <= R.bf16(b))


@pytest.fixture(scope="module")
def step(oracle_window):  # noqa: F811
    p, s0, s1, t0, dt, W = oracle_window
    T = W * dt
    act = _act(p, t0, T)
    sur, params, scales = _setup_network(p, s0, s1, act, T)
    loss = sur.train_step(_cuda(s0), _cuda(s1), _cuda([act])[0], lr=0.0)
    bufs = {k: sur.debug_buffer(k).astype(np.float64) for k in range(13)}
    layers = R.unpack(params)
    Wb = [(R.bf16(Wl), bl.astype(np.float32).astype(np.float64)) for Wl, bl in layers]
    return {"loss": loss, "grad": sur.get_grad().astype(np.float64), "bufs": bufs, "W": Wb,
            "params": params, "scales": scales, "s0": s0, "act": act}


def _check_pre(z_gpu, inp, W, b, K):
    z = R.conv(inp, W, b)
    mag = R.conv(np.abs(inp), np.abs(W), np.abs(b))
    err = np.abs(z_gpu - z)
    bound = (K + 2) * U22 * mag + 1e-37
    assert np.all(err <= bound), (float((err / np.maximum(mag, 1e-300)).max()), K)
    return float((err / np.maximum(mag, 1e-300)).max())


def _feature_bracket(F, M, x, sh, sc):
    """[lo, hi] for every network input entry: (raw - shift) * float32(scale) from the reference
    raw features F (FP64), widened by a bound on the kernels' FP32 evaluation error, rounded to
    BF16 at both ends (rounding is monotone), zero where a feature is undefined.

    The kernels form each raw value v in FP32 from the FP64 state, subtract the shift rounded to
    FP32 and multiply by the FP32 scale.  Bounds on |v_fp32 - v| (u = 2^-24, one FP32 rounding):
    state values (velocity, directors, angular velocity, base couple) u |v|; the position
    relative to the base, a difference of two rounded positions, 3u (|x_j| + |x_0|); the relative
    rotation, half a difference of two 3-term dot products of rounded unit vectors, below
    (2 + 3) u sqrt(3) < 2^-19; the edge Q_j l with l the FP64 difference rounded once, below
    2^-19 |l| (|l| = |Q_j l| from the reference).  To that the shift's rounding (u |shift|) and the
    two roundings of the subtraction and the product (2u of their results)."""
    nwin = F.shape[0]
    X = np.asarray(x, dtype=np.float64).reshape(3, nwin, R.POS).transpose(1, 0, 2)   # (nwin, 3, 51)
    shv = np.asarray(sh, dtype=np.float64)[None, :, None]
    sc32 = np.abs(np.asarray(sc, dtype=np.float64).astype(np.float32).astype(np.float64))[None, :, None]
    u = 2.0 ** -24
    e = np.zeros_like(F)
    e[:, 0:3] = 3 * u * (np.abs(X) + np.abs(X[:, :, :1]))
    e[:, 3:15] = u * np.abs(F[:, 3:15])
    e[:, 21:24] = u * np.abs(F[:, 21:24])
    e[:, 15:18] = 2.0 ** -19
    e[:, 18:21] = 2.0 ** -19 * np.sqrt((F[:, 18:21] ** 2).sum(axis=1, keepdims=True))
    exact = (F - shv) * np.asarray(sc, dtype=np.float64).astype(np.float32)[None, :, None]
    E = sc32 * (e + u * np.abs(shv) + 2 * u * (np.abs(F - shv) + e)) + 2 * u * np.abs(exact)
    lo = np.where(M, R.bf16(exact - E), 0.0)
    hi = np.where(M, R.bf16(exact + E), 0.0)
    return lo, hi


def test_network_input_is_the_bf16_rounding_of_the_reference_features(step, oracle_window):  # noqa: F811
    """The training path's network input (features_kernel): every entry is the BF16 rounding of
    a value within the FP32 evaluation bound of (raw - shift) * scale (_feature_bracket); the
    padding rows and channels 24..31 are zero."""
    sh, sc, _ = step["scales"]
    F, M = R.raw_features(*step["s0"], step["act"])
    lo, hi = _feature_bracket(F, M, step["s0"][0], sh, sc)
    got = _cp(step["bufs"][0])
    assert np.all(got[:, R.N_FEAT:] == 0.0)
    g = got[:, :R.N_FEAT]
    ok = (lo <= g) & (g <= hi)
    assert np.all(ok), np.argwhere(~ok)[:5].tolist()
    pad = step["bufs"][0]
    assert np.all(pad[:, :2] == 0) and np.all(pad[:, 2 + R.POS:] == 0)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_hidden_layer_pre_activations_and_activations(step, layer):
    bufs = step["bufs"]
    Wl, bl = step["W"][layer]
    inp = _cp(bufs[layer])
    K = R.TAPS * inp.shape[1]
    pre = _cp(bufs[4 + layer])
    _check_pre(pre, inp, Wl, bl, K)
    # activation: BF16 of the FP32 SiLU of the FP32 pre-activation
    s = R.silu(pre)
    eps = _silu_rel(pre)
    got = _cp(bufs[layer + 1])
    ok = _bf16_bracket(got, s - eps * np.abs(s) - _silu_abs(pre), s + eps * np.abs(s) + _silu_abs(pre))
    assert np.all(ok), int((~ok).sum())
    out = bufs[layer + 1]
    assert np.all(out[:, :2] == 0) and np.all(out[:, 2 + R.POS:] == 0)


def test_output_layer(step):
    bufs = step["bufs"]
    W4, b4 = step["W"][3]
    out = np.asarray(bufs[7], dtype=np.float64).transpose(0, 2, 1)        # [nwin, 16, 51]
    _check_pre(out, _cp(bufs[3]), W4, b4, R.TAPS * 64)


def test_loss_and_its_gradient(step):
    bufs = step["bufs"]
    out = bufs[7][:, :, :R.N_OUT]
    tgt = bufs[8][:, :, :R.N_OUT]
    r = out - tgt
    n = r.size
    ref = float((r * r).sum() / n)
    assert abs(step["loss"] - ref) <= (n + 4) * U23 * ref, (step["loss"], ref)
    g = 2.0 * r / n
    eps = 4 * 2.0 ** -24
    got = bufs[9][:, 2:2 + R.POS, :R.N_OUT]
    assert np.all(_bf16_bracket(got, g - eps * np.abs(g), g + eps * np.abs(g)))
    assert np.all(bufs[9][:, :, R.N_OUT:] == 0) and np.all(bufs[9][:, :2] == 0) and np.all(bufs[9][:, 2 + R.POS:] == 0)


@pytest.mark.parametrize("layer", [3, 2, 1])
def test_back_propagated_gradients(step, layer):
    """g at the output of layer `layer` (1-based below it) from the gradient above: the input
    gradient of the convolution, times SiLU' of the lower pre-activation, stored in BF16."""
    bufs = step["bufs"]
    W, _ = step["W"][layer]
    g_above = _cp(bufs[9 + (3 - layer)])          # 9: output gradient, 10: layer 3's, 11: layer 2's
    acc = R.conv_input_grad(g_above, W)
    mag = R.conv_input_grad(np.abs(g_above), np.abs(W))
    K = R.TAPS * g_above.shape[1]
    B = (K + 2) * U22 * mag + 1e-38
    x = _cp(bufs[4 + layer - 1])                  # pre-activation of the layer below
    d = R.dsilu(x)
    ed = (2.0 ** -21) * (1.0 + np.abs(x)) * (3.0 + 1.2 * np.abs(x)) * np.maximum(1.0, np.abs(d))
    corners = [(acc + sa * B) * (d + sd * ed) for sa in (-1, 1) for sd in (-1, 1)]
    lo = np.minimum.reduce(corners)
    hi = np.maximum.reduce(corners)
    lo, hi = lo - 2.0 ** -24 * np.abs(lo) - 1e-38, hi + 2.0 ** -24 * np.abs(hi) + 1e-38
    got = _cp(bufs[10 + (3 - layer)])
    ok = _bf16_bracket(got, lo, hi)
    assert np.all(ok), int((~ok).sum())


@pytest.mark.parametrize("layer", [0, 1, 2, 3])
def test_weight_and_bias_gradients(step, layer):
    bufs = step["bufs"]
    g = _cp(bufs[9 + (3 - layer)])                # gradient at the output of this layer
    a = _cp(bufs[layer])                          # its input activations
    dW, db = R.conv_weight_grad(g, a)
    mW, mb = R.conv_weight_grad(np.abs(g), np.abs(a))
    nwin = g.shape[0]
    M = min(nwin, 16) * 64 + (nwin + 15) // 16
    off = 0
    for l, (co, ci) in enumerate(R.SHAPES):
        if l == layer:
            break
        off += co * R.TAPS * ci + co
    co, ci = R.SHAPES[layer]
    gw = step["grad"][off:off + co * R.TAPS * ci].reshape(co, R.TAPS, ci)
    gb = step["grad"][off + co * R.TAPS * ci:off + co * R.TAPS * ci + co]
    assert np.all(np.abs(gw - dW) <= (M + 4) * U22 * mW + 1e-38), float((np.abs(gw - dW) / np.maximum(mW, 1e-300)).max())
    assert np.all(np.abs(gb - db) <= (M + 4) * U22 * mb + 1e-38)
    assert np.abs(dW).max() > 0


# ---- the fused inference kernel (tcgen05 tensor cores): the same checks on its captured arrays

@pytest.fixture(scope="module", params=["oracle_9_rods", "carpet_5x5", "carpet_40x40"])
def tc_call(oracle_window, request):  # noqa: F811
    """One window call of the fused kernel, with every layer's arrays captured: on the oracle's
    windows (9 rods, one full group of nine), on a perturbed 5 x 5 carpet (25 rods: groups of
    9, 9 and 7, the last with two empty window slots) and on a perturbed 40 x 40 carpet (1600
    rods: 178 groups, more than one per block of the persistent grid)."""
    from paper_2605_13766_gb300 import RodSystem
    p, s0, s1, t0, dt, W = oracle_window
    T = W * dt
    act = _act(p, t0, T)
    sur, params, scales = _setup_network(p, s0, s1, act, T)
    if request.param != "oracle_9_rods":
        side = 5 if request.param == "carpet_5x5" else 40
        p = rodgen.perturbed(rodgen.cilia_carpet(side=side, n=50), seed=side, pos=0.01, vel=0.02, rot=0.02,
                             omega=1.0)
        s0 = p.state()
        act = _act(p, t0, T)
    s = RodSystem(p)
    s.set_state(*s0)
    s.time = t0
    pre, inp = sur.apply_debug(s)
    new_state = s.get_state()
    s.close()
    layers = R.unpack(params)
    Wb = [(R.bf16(Wl), bl.astype(np.float32).astype(np.float64)) for Wl, bl in layers]
    tr = lambda a: np.asarray(a, dtype=np.float64).transpose(0, 2, 1)   # [R, 51, 64] -> [R, 64, 51]
    return {"pre": [tr(pre[l]) for l in range(4)], "inp": [tr(inp[l]) for l in range(4)], "W": Wb,
            "scales": scales, "s0": s0, "act": act, "new": new_state, "T": T, "clamp": p.clamp_base}


def test_tensor_core_input_features(tc_call):
    """The fused kernel's network input, against the same bracket as the training path's."""
    sh, sc, _ = tc_call["scales"]
    F, M = R.raw_features(*tc_call["s0"], tc_call["act"])
    lo, hi = _feature_bracket(F, M, tc_call["s0"][0], sh, sc)
    got = tc_call["inp"][0]
    assert np.all(got[:, R.N_FEAT:32] == 0.0)
    g = got[:, :R.N_FEAT]
    ok = (lo <= g) & (g <= hi)
    assert np.all(ok), np.argwhere(~ok)[:5].tolist()


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_tensor_core_hidden_layers(tc_call, layer):
    Wl, bl = tc_call["W"][layer]
    cin = Wl.shape[2]
    inp = tc_call["inp"][layer][:, :cin]
    pre = tc_call["pre"][layer]
    _check_pre(pre, inp, Wl, bl, R.TAPS * cin)
    s = R.silu(pre)
    eps = _silu_rel(pre)
    got = tc_call["inp"][layer + 1]
    ok = _bf16_bracket(got, s - eps * np.abs(s) - _silu_abs(pre), s + eps * np.abs(s) + _silu_abs(pre))
    bad = ~ok
    assert np.all(ok), (int(bad.sum()), np.percentile(pre[bad], [0, 50, 100]).tolist(), got[bad][:5].tolist(),
                        s[bad][:5].tolist())


def test_tensor_core_output_layer_and_update(tc_call):
    W4, b4 = tc_call["W"][3]
    out = tc_call["pre"][3][:, :16]
    _check_pre(out, tc_call["inp"][3], W4, b4, R.TAPS * 64)
    # the FP64 update from the kernel's own outputs, as the reference computes it
    _, _, out_scale = tc_call["scales"]
    ref = R.apply(tc_call["s0"], out.transpose(0, 2, 1), out_scale, tc_call["T"], tc_call["clamp"])
    for a, b in zip(tc_call["new"], ref):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1.0)
