"""Learned window surrogate on the GPU: its kernels against the numpy reference of the same
network (oracle side), then training, the checked rollout and the fallback.

Parity cases use windows of the CPU oracle (3 x 3 carpet of 50-element rods, bent by 400 steps
of actuation, then one window of 50 steps).  Tolerances:
  * unscaled features and targets (FP64 on both sides): 1e-12 of each channel's magnitude;
  * network output, loss and gradient of the whole network against the reference, which rounds
    to BF16 at every point the kernels store BF16 (an end-to-end cross-check; the element-wise
    parity of every layer is in test_gpu_surrogate_layers.py): what remains is FP32 versus FP64
    accumulation and the rare BF16 rounding it flips, which then propagates through the later
    layers: 2e-3 (output, norm-wise), 2e-3 (loss), 2e-2 (gradient per layer, norm-wise);
  * state update (FP64 on both sides, same network outputs): 1e-12.
"""
import json
import os
import time

import numpy as np
import pytest

import rodgen
from oracle import surrogate_ref as R
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _record(name, obj):
    """Write obj as JSON into the directory named by ROD_TEST_RECORD_DIR, when it is set."""
    out = os.environ.get("ROD_TEST_RECORD_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, f"{name}.json"), "w") as f:
            json.dump(obj, f, indent=1)


@pytest.fixture(scope="module")
def oracle_window():
    p = rodgen.cilia_carpet(side=3, n=50, amp_range=(0.3, 0.8), period_range=(0.05, 0.2), seed=11)
    dt, W = 1e-5, 50
    o = Oracle(p)
    s0 = o.step(*p.state(), dt=dt, n_steps=400)
    t0 = 400 * dt
    s1 = o.step(*s0, dt=dt, n_steps=W, t=t0)
    return p, s0, s1, t0, dt, W


def _act(p, t0, T):
    from paper_2605_13766_gb300.surrogate import couple_samples
    return couple_samples(p, t0, T)


def _cuda(arrs):
    import torch
    return [torch.tensor(np.ascontiguousarray(a), device="cuda") for a in arrs]


def _scales(F, M, D):
    from paper_2605_13766_gb300.surrogate import scales_from_moments
    mean = np.array([F[:, c][M[:, c]].mean() for c in range(R.N_FEAT)])
    std = np.array([F[:, c][M[:, c]].std() for c in range(R.N_FEAT)])
    rms = np.sqrt((D ** 2).mean(axis=(0, 2)))
    return scales_from_moments(mean, std, rms)


def test_raw_features_and_targets_match_reference(oracle_window):
    from paper_2605_13766_gb300 import Surrogate
    p, s0, s1, t0, dt, W = oracle_window
    act = _act(p, t0, W * dt)
    sur = Surrogate(W, dt)
    Fg, Mg = sur.raw_features(_cuda(s0), _cuda([act])[0])
    F, M = R.raw_features(*s0, act)
    assert np.array_equal(Mg.cpu().numpy().astype(bool), M)
    Fg = Fg.cpu().numpy()
    for c in range(R.N_FEAT):
        mag = max(np.abs(F[:, c]).max(), 1e-300)
        assert np.abs(Fg[:, c] - F[:, c]).max() <= 1e-12 * mag, c
    Dg = sur.raw_targets(_cuda(s0), _cuda(s1)).cpu().numpy()
    D = R.raw_targets(s0, s1, W * dt)
    # a target is a difference of state entries: beside 1e-12 of the channel, allow a few ulps of
    # the entries it is taken from (a channel that is zero up to rounding is rounding on both sides)
    operand = [np.abs(s1[0]).max()] * 3 + [np.abs(s1[1]).max()] * 3 + [1.0] * 6 + [np.abs(s1[3]).max()] * 3
    for c in range(R.N_OUT):
        mag = np.abs(D[:, c]).max()
        assert np.abs(Dg[:, c] - D[:, c]).max() <= 1e-12 * mag + 4e-16 * operand[c], c


def _setup_network(p, s0, s1, act, T, seed=3):
    from paper_2605_13766_gb300 import Surrogate
    from paper_2605_13766_gb300.surrogate import initial_params
    F, M = R.raw_features(*s0, act)
    D = R.raw_targets(s0, s1, T)
    sh, sc, out = _scales(F, M, D)
    params = initial_params(seed=seed, last_gain=1.0).astype(np.float64)
    rng = np.random.default_rng(seed)
    # non-zero biases so that their gradients and the bias path are exercised
    for off, n in _bias_blocks():
        params[off:off + n] = rng.normal(0, 0.1, n)
    params = params.astype(np.float32)
    sur = Surrogate(50, T / 50)
    sur.set_params(params)
    sur.set_scales(sh, sc, out)
    return sur, params.astype(np.float64), (sh, sc, out)


def _bias_blocks():
    off, blocks = 0, []
    for co, ci in R.SHAPES:
        off += co * R.TAPS * ci
        blocks.append((off, co))
        off += co
    return blocks


def test_forward_matches_bf16_reference(oracle_window):
    p, s0, s1, t0, dt, W = oracle_window
    T = W * dt
    act = _act(p, t0, T)
    sur, params, (sh, sc, out_sc) = _setup_network(p, s0, s1, act, T)
    got = sur.forward(_cuda(s0), _cuda([act])[0]).cpu().numpy()          # (nwin, 51, 16)
    feats = R.features(*s0, act, sh, sc, emulate=True)
    ref, _ = R.forward(params, feats, emulate=True)                       # (nwin, 16, 51)
    ref64, _ = R.forward(params, R.features(*s0, act, sh, sc, emulate=False), emulate=False)
    g = got.transpose(0, 2, 1)[:, :R.N_OUT]
    r = ref[:, :R.N_OUT]
    err = np.linalg.norm(g - r) / np.linalg.norm(r)
    err64 = np.linalg.norm(g - ref64[:, :R.N_OUT]) / np.linalg.norm(r)
    _record("surrogate_forward_parity", {"rel_err_vs_bf16_reference": err, "rel_err_vs_fp64_reference": err64})
    assert err <= 2e-3, (err, err64)


def test_train_step_loss_and_gradient_match_reference(oracle_window):
    p, s0, s1, t0, dt, W = oracle_window
    T = W * dt
    act = _act(p, t0, T)
    sur, params, (sh, sc, out_sc) = _setup_network(p, s0, s1, act, T)
    loss = sur.train_step(_cuda(s0), _cuda(s1), _cuda([act])[0], lr=0.0)
    grad = sur.get_grad().astype(np.float64)
    feats = R.features(*s0, act, sh, sc, emulate=True)
    tg = R.targets(s0, s1, out_sc, T)
    loss_ref, grad_ref = R.loss_and_grad(params, feats, tg, emulate=True)
    loss64, grad64 = R.loss_and_grad(params, R.features(*s0, act, sh, sc, emulate=False), tg, emulate=False)
    rows = {"loss": loss, "loss_ref": loss_ref, "loss_fp64": loss64}
    assert abs(loss - loss_ref) <= 2e-3 * loss_ref, rows
    off = 0
    for l, (co, ci) in enumerate(R.SHAPES):
        for name, n in (("W", co * R.TAPS * ci), ("b", co)):
            g, gr = grad[off:off + n], grad_ref[off:off + n]
            e = float(np.linalg.norm(g - gr) / np.linalg.norm(gr))
            rows[f"{name}{l + 1}_rel_err"] = e
            rows[f"{name}{l + 1}_rel_err_fp64"] = float(np.linalg.norm(g - grad64[off:off + n]) / np.linalg.norm(gr))
            assert e <= 2e-2, (l, name, rows)
            off += n
    _record("surrogate_gradient_parity", rows)
    # and the optimiser moves the parameters against the gradient
    before = sur.get_params()
    sur.train_step(_cuda(s0), _cuda(s1), _cuda([act])[0], lr=1e-3)
    step = sur.get_params() - before
    assert float(np.dot(step, grad)) < 0


def test_apply_matches_reference_update(oracle_window):
    import torch
    from paper_2605_13766_gb300 import RodSystem
    p, s0, s1, t0, dt, W = oracle_window
    T = W * dt
    q = p.replace(act_amp=np.zeros(p.n_rods))          # couple features exactly zero on both sides
    act = np.zeros((3, q.n_rods))
    sur, params, (sh, sc, out_sc) = _setup_network(q, s0, s1, act, T)
    out = sur.forward(_cuda(s0), _cuda([act])[0]).cpu().numpy()
    ref = R.apply(s0, out, out_sc, T, q.clamp_base.astype(bool))
    s = RodSystem(q)
    s.set_state(*s0)
    sur.apply(s, 1)
    got = s.get_state()
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1.0)
    assert abs(s.time - T) < 1e-15


def test_fused_tensor_core_inference_agrees_with_the_unfused_kernels(oracle_window, monkeypatch):
    """The fused inference kernel (tcgen05 tensor cores) and the kernel-by-kernel path (mma.sync)
    sum the same BF16 products in different orders, so a BF16 rounding may flip between them
    and the two states differ by a little of the network's correction; two calls on a perturbed
    6 x 6 carpet: the learned part of the new positions and velocities (state minus the
    kinematic prior) agrees to 2 % of its size.  The element-wise parity of every layer of the
    fused kernel is in test_gpu_surrogate_layers.py."""
    from paper_2605_13766_gb300 import RodSystem
    p, s0, s1, t0, dt, W = oracle_window
    act = _act(p, t0, W * dt)
    sur, params, _ = _setup_network(p, s0, s1, act, W * dt)
    q = rodgen.perturbed(rodgen.cilia_carpet(side=6, n=50), seed=4, pos=0.01, vel=0.02, rot=0.02, omega=1.0)
    results = {}
    for mode, env in (("unfused", {"ROD_SURROGATE_UNFUSED": "1"}), ("fused", {})):
        monkeypatch.delenv("ROD_SURROGATE_UNFUSED", raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        s = RodSystem(q)
        s.set_state(*q.state())
        s.time = 0.0123
        sur.apply(s, 1)
        results[mode] = s.get_state()
        s.close()
    T = W * dt
    x0, v0 = q.state()[0], q.state()[1]
    for idx, prior in ((0, x0 + T * v0), (1, v0)):
        learned = results["unfused"][idx] - prior
        diff = results["fused"][idx] - results["unfused"][idx]
        assert np.abs(learned).max() > 0
        assert np.abs(diff).max() <= 2e-2 * np.abs(learned).max(), (idx, np.abs(diff).max(), np.abs(learned).max())


def test_a_tensor_core_wait_that_runs_out_is_reported(oracle_window):
    """With the test hook the fused kernel issues no MMA, its bounded wait runs out, it latches
    ROD_ERR_TIMEOUT, frees its tensor memory and ends without touching the state; afterwards the
    same surrogate and system run normally."""
    from paper_2605_13766_gb300 import RodError, RodSystem
    p, s0, s1, t0, dt, W = oracle_window
    act = _act(p, t0, W * dt)
    sur, params, _ = _setup_network(p, s0, s1, act, W * dt)
    q = rodgen.cilia_carpet(side=6, n=50)
    s = RodSystem(q)
    s.set_state(*q.state())
    sur.set_wait_polls(0x80000000 | 1000)
    with pytest.raises(RodError) as ei:
        sur.apply(s, 1)
    assert ei.value.status == -4
    x_after = s.get_state()[0]
    assert np.array_equal(x_after, q.x)
    sur.set_wait_polls(0)
    s.set_state(*q.state())                       # clears the error word
    sur.apply(s, 2)
    assert np.all(np.isfinite(s.get_state()[0])) and not np.array_equal(s.get_state()[0], q.x)
    s.close()


# ---- training on windows of the plain GPU step, checked rollout, fallback


def _carpet_eval(side=64):
    return rodgen.cilia_carpet(side=side, n=50)


@pytest.fixture(scope="module")
def trained():
    """A network trained on 2 x 10^5 windows of a carpet with random amplitude, period and phase."""
    from paper_2605_13766_gb300 import surrogate as S
    t = time.time()
    sur, info = S.train_default(steps=int(os.environ.get("ROD_SURROGATE_TRAIN_STEPS", "15000")))
    info["total_s"] = time.time() - t
    return sur, info


def test_trained_surrogate_gain_over_plain_step(trained):
    """The 64 x 64 carpet of 50-element rods from rest over 10^4 fine steps (200 calls): the
    trained network's tip error stays within 1e-3 L at every 20th call, and the checked rollout
    (sampled rods against a shadow system every 10 calls) is faster than the plain step."""
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300 import surrogate as S
    sur, info = trained
    p = _carpet_eval()
    dt, W, n_calls = 1e-5, 50, 200
    # plain GPU step: reference states every 20 calls, then the same run timed without stops
    s = RodSystem(p)
    s.set_state(*p.state())
    ref = {}
    for k in range(1, 11):
        s.step(20 * W, dt)
        ref[20 * k] = s.get_state()[0]
    s.set_state(*p.state())
    s.step(W, dt)
    s.set_state(*p.state())
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.step(n_calls * W, dt)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t
    s.close()
    # the network alone, compared every 20 calls
    net = RodSystem(p)
    net.set_state(*p.state())
    curve = {}
    for k in range(1, 11):
        sur.apply(net, 20)
        e = S.tip_error(p, net.get_state()[0], ref[20 * k])
        d = S.tip_error(p, ref[20 * k], p.x)
        curve[20 * k] = {"max_err": float(e.max()), "mean_err": float(e.mean()), "plain_disp_max": float(d.max())}
    net.close()
    # checked rollouts (global and local checks), timed
    el_steps = p.n_elems * n_calls * W
    worst = max(v["max_err"] for v in curve.values())
    rec = dict(info, plain_s=t_plain, plain_elem_steps_per_s=el_steps / t_plain, network_curve=curve,
               network_worst_tip_err=worst)
    for mode in ("global", "local"):
        warm = S.CheckedRollout(sur, p, seed=1, mode=mode)
        warm.run(2, check_every=1, bound=1.0)
        warm.close()
        ro = S.CheckedRollout(sur, p, seed=1, mode=mode)
        torch.cuda.synchronize()
        t = time.perf_counter()
        stats = ro.run(n_calls, check_every=10, bound=S.DEFAULT_CHECK_BOUND)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t
        err = S.tip_error(p, ro.system.get_state()[0], ref[n_calls])
        ro.close()
        rec[mode] = dict(rollout_s=t_sur, speedup=t_plain / t_sur, rollout_elem_steps_per_s=el_steps / t_sur,
                         final_tip_err=float(err.max()), stats=stats)
        assert err.max() <= 1e-3, rec
        # what the trained network gains: at least 10x the plain step with the pipelined local
        # checks; the global check follows sampled rods with sequential plain steps on a shadow
        # system, which bounds it near 9x, so it must only beat the plain step
        assert t_plain / t_sur >= (10.0 if mode == "local" else 1.0), rec
    assert worst <= 1e-3, rec                             # the bound, every 20th call, all 4096 rods
    # out of the training window: t in [0.5, 0.6] s of the same carpet (no training window
    # covers it), and a carpet whose amplitude and period lie outside the training ranges,
    # where the checks must take over (fallbacks) and keep the bound
    later = _advanced(p, dt, 50_000)
    rec["t_0.5_to_0.6_s"] = _checked_case(sur, later, dt, W, n_calls, t0=0.5)
    assert rec["t_0.5_to_0.6_s"]["final_tip_err"] <= 1e-3, rec
    assert rec["t_0.5_to_0.6_s"]["speedup"] >= 10.0, rec
    beyond = rodgen.cilia_carpet(side=64, n=50, amp_factor=1.0, period=0.3)
    rec["amp_1.0_period_0.3"] = _checked_case(sur, beyond, dt, W, n_calls)
    assert rec["amp_1.0_period_0.3"]["final_tip_err"] <= 1e-3, rec
    assert rec["amp_1.0_period_0.3"]["fallback_calls"] > 0, rec
    _record("surrogate_gain", rec)
    print(json.dumps(rec, indent=1))


def _advanced(p, dt, n_steps):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    s.step(n_steps, dt)
    x, v, Q, w = s.get_state()
    s.close()
    return p.replace(x=x, v=v, Q=Q, w=w)


def _local_segments(n_calls, every):
    """The local checks' segment lengths as rod_surrogate_rollout_local documents them: every
    calls each, except toward the end, where a segment has a third of the calls after it (at
    least one)."""
    after, tail = 0, []
    while after < n_calls:
        L = max(1, min(every, after // 3))
        if L == every:
            break
        L = min(L, n_calls - after)
        tail.append(L)
        after += L
    head = n_calls - after
    return [min(every, head - d) for d in range(0, head, every)] + tail[::-1]


def _checked_case(sur, p, dt, W, n_calls, t0=0.0):
    """Checked rollout with local checks from the problem's state at time t0 against the plain
    GPU step over the same interval (wall clock around each, after a synchronisation)."""
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300 import surrogate as S
    s = RodSystem(p)
    s.set_state(*p.state())
    s.time = t0
    s.step(W, dt)                                           # warm-up
    s.set_state(*p.state())
    s.time = t0
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.step(n_calls * W, dt)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t
    ref = s.get_state()[0]
    s.close()
    ro = S.CheckedRollout(sur, p, seed=1, mode="local", t0=t0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    stats = ro.run(n_calls, check_every=10, bound=S.DEFAULT_CHECK_BOUND)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t
    err = S.tip_error(p, ro.system.get_state()[0], ref)
    ro.close()
    return {"speedup": t_plain / t_sur, "final_tip_err": float(err.max()),
            "fallback_calls": int(stats["fallback_calls"]), "surrogate_calls": int(stats["surrogate_calls"])}


@pytest.mark.parametrize("mode", ["global", "local"])
def test_untrained_network_falls_back_to_the_plain_step(mode):
    """With random weights every checked segment exceeds the bound, is undone and redone with
    the plain step: the result is the plain trajectory."""
    import torch
    from paper_2605_13766_gb300 import RodSystem, Surrogate
    from paper_2605_13766_gb300 import surrogate as S
    p = rodgen.cilia_carpet(side=8, n=50)
    dt, W, n_calls, every = 1e-5, 50, 20, 5
    sur = Surrogate(W, dt)
    sur.set_params(S.initial_params(seed=5, last_gain=1.0))
    sur.set_scales(np.zeros(24), np.ones(24), np.full(15, 1e-3))
    ro = S.CheckedRollout(sur, p, n_sample=8, seed=2, mode=mode, n_shadows=3)
    stats = ro.run(n_calls, check_every=every, bound=1e-3)
    assert stats["fallback_calls"] == n_calls and stats["surrogate_calls"] == 0, stats
    segments = [every] * (n_calls // every) if mode == "global" else _local_segments(n_calls, every)
    assert stats["checks"] == len(segments) and stats["rejected_err"] > 1e-3, stats
    # the plain step in the same calls as the redone segments (a call's kinematic half steps at
    # its ends round differently from the fused full steps inside it)
    s = RodSystem(p)
    s.set_state(*p.state())
    for L in segments:
        s.step(L * W, dt)
    for a, b in zip(ro.system.get_state(), s.get_state()):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1.0)
    assert stats["max_err"] < 1e-12
    ro.close()


def _perturb_reference(state, draws, spread, noise, held):
    """NumPy statement of the noise-injected window start: additive noise on x, v, w, a
    first-order lab-frame turn d_a + ang x d_a of d1 and d2 with ang = noise x (largest director
    spread) x draw, Gram-Schmidt, d3 = d1 x d2, and the held windows' node 0 and element 0 kept."""
    x, v, Q, w = [np.array(a, dtype=np.float64) for a in state]
    rx, rv, rw, ra = [np.asarray(a, dtype=np.float64) for a in draws]
    sp = np.asarray(spread, dtype=np.float64)
    nwin = x.shape[1] // R.POS
    xo = x + noise * sp[0:3, None] * rx
    vo = v + noise * sp[3:6, None] * rv
    wo = w + noise * sp[12:15, None] * rw
    ang = noise * sp[6:12].max() * ra
    d1 = Q[0:3] + np.cross(ang, Q[0:3], axis=0)
    d2 = Q[3:6] + np.cross(ang, Q[3:6], axis=0)
    d1 = d1 / np.linalg.norm(d1, axis=0)
    d2 = d2 - (d1 * d2).sum(axis=0) * d1
    d2 = d2 / np.linalg.norm(d2, axis=0)
    Qo = np.concatenate([d1, d2, np.cross(d1, d2, axis=0)])
    for b in np.flatnonzero(held):
        n, e = b * R.POS, b * (R.POS - 1)
        xo[:, n] = x[:, n]
        vo[:, n] = 0.0
        Qo[:, e] = Q[:, e]
        wo[:, e] = 0.0
    return xo, vo, Qo, wo


@pytest.mark.parametrize("noise", [0.05, 0.0])
def test_training_perturbation_kernel_matches_its_statement(oracle_window, noise):
    """The training's noise-injected window start (rod_surrogate_perturb) against its NumPy
    statement on the oracle window's perturbed states, with two of the nine windows held; at
    zero noise it only re-orthonormalises the directors (given slightly off-orthonormal)."""
    import torch
    from paper_2605_13766_gb300 import Surrogate
    p, s0, s1, t0, dt, W = oracle_window
    rng = np.random.default_rng(8)
    x, v, Q, w = [np.array(a, dtype=np.float64) for a in s0]
    Q = Q + 1e-6 * rng.normal(size=Q.shape)          # off SO(3) by a little
    draws = [rng.normal(size=x.shape), rng.normal(size=v.shape), rng.normal(size=w.shape), rng.normal(size=w.shape)]
    spread = np.abs(rng.normal(size=15)) * 1e-3 + 1e-4
    held = np.zeros(x.shape[1] // R.POS, dtype=np.int8)
    held[[0, 4]] = 1
    sur = Surrogate(W, dt)
    got = sur.perturb(_cuda([x, v, Q, w]), _cuda(draws), spread, noise, torch.tensor(held, device="cuda"))
    ref = _perturb_reference((x, v, Q, w), draws, spread, noise, held)
    for g, r in zip(got, ref):
        g = g.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-14 * max(np.abs(r).max(), 1.0)
    Qg = got[2].cpu().numpy()
    d1, d2, d3 = Qg[0:3], Qg[3:6], Qg[6:9]
    free = np.ones(Qg.shape[1], dtype=bool)
    free[[0, 4 * (R.POS - 1)]] = False
    for a, b, want in ((d1, d1, 1.0), (d2, d2, 1.0), (d3, d3, 1.0), (d1, d2, 0.0), (d1, d3, 0.0)):
        assert np.abs((a * b).sum(axis=0)[free] - want).max() <= 1e-15
