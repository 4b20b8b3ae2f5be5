"""Plain numpy reference of the learned surrogate's network, loss and gradient.

TEST INFRASTRUCTURE ONLY.  FP64 forward and hand-derived backward of the four 1D convolutions
(kernel 5, zero padding, SiLU) that the CUDA surrogate evaluates with BF16 tensor cores, plus
the features, targets and state update it is trained and applied with.  With ``emulate=True`` every quantity the GPU stores
in BF16 (features, weights, hidden activations, back-propagated gradients) is rounded to BF16
at the same point, so that the remaining difference is FP32 versus FP64 accumulation.

Parameter vector layout (FP32 on the GPU): W1 [64][5][32], b1 [64], W2 [64][5][64], b2 [64],
W3 [64][5][64], b3 [64], W4 [16][5][64], b4 [16] (W[o, t, c] multiplies input channel c at
position p + t - 2 for output position p).
"""
from __future__ import annotations

import numpy as np

POS = 51
TAPS = 5
SHAPES = [(64, 32), (64, 64), (64, 64), (16, 64)]   # (C_out, C_in) per layer
N_FEAT, N_OUT = 24, 15


def n_params() -> int:
    return sum(co * TAPS * ci + co for co, ci in SHAPES)


def unpack(params):
    out, off = [], 0
    for co, ci in SHAPES:
        W = np.asarray(params[off:off + co * TAPS * ci], dtype=np.float64).reshape(co, TAPS, ci)
        off += co * TAPS * ci
        b = np.asarray(params[off:off + co], dtype=np.float64)
        off += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def conv(inp, W, b):
    """out[n, o, p] = b[o] + sum_{t,c} W[o, t, c] inp[n, c, p + t - 2] (zero outside 0..50)."""
    n, ci, P = inp.shape
    pad = np.zeros((n, ci, P + 4))
    pad[:, :, 2:P + 2] = inp
    out = np.zeros((n, W.shape[0], P)) + b[None, :, None]
    for t in range(TAPS):
        out += np.einsum("oc,ncp->nop", W[:, t, :], pad[:, :, t:t + P])
    return out


def conv_input_grad(g, W):
    """d(loss)/d(inp) of conv: gin[n, c, p] = sum_{o,t} W[o, t, c] g[n, o, p - t + 2]."""
    n, co, P = g.shape
    pad = np.zeros((n, co, P + 4))
    pad[:, :, 2:P + 2] = g
    gin = np.zeros((n, W.shape[2], P))
    for t in range(TAPS):
        gin += np.einsum("oc,nop->ncp", W[:, t, :], pad[:, :, 4 - t:4 - t + P])
    return gin


def conv_weight_grad(g, inp):
    """dW[o, t, c] = sum_{n,p} g[n, o, p] inp[n, c, p + t - 2]; db[o] = sum g."""
    n, ci, P = inp.shape
    pad = np.zeros((n, ci, P + 4))
    pad[:, :, 2:P + 2] = inp
    dW = np.stack([np.einsum("nop,ncp->oc", g, pad[:, :, t:t + P]) for t in range(TAPS)], axis=1)
    return dW, g.sum(axis=(0, 2))


def _split(x, v, Q, w, nwin):
    X = x.reshape(3, nwin, POS)
    V = v.reshape(3, nwin, POS)
    Qm = Q.reshape(3, 3, nwin, POS - 1)        # Qm[a, k]: component k of director a
    We = w.reshape(3, nwin, POS - 1)
    return X, V, Qm, We


def raw_features(x, v, Q, w, act):
    """(nwin, 24, 51) raw features and a mask of where each is defined.

    Channels: 0..2 node position minus the base node, 3..5 node velocity, 6..11 directors d1, d2
    of element j, 12..14 angular velocity of element j, 15..17 half the axial vector of R - R^T
    for R = Q_j Q_{j-1}^T (Voronoi points 1..49), 18..20 the edge Q_j (x_{j+1} - x_j), 21..23 the
    base couple at the window's start, middle and end (act rows)."""
    nwin = act.shape[1]
    X, V, Qm, We = _split(x, v, Q, w, nwin)
    F = np.zeros((nwin, N_FEAT, POS))
    M = np.zeros((nwin, N_FEAT, POS), dtype=bool)
    F[:, 0:3, :] = (X - X[:, :, :1]).transpose(1, 0, 2)
    F[:, 3:6, :] = V.transpose(1, 0, 2)
    M[:, 0:6, :] = True
    F[:, 6:9, :POS - 1] = Qm[0].transpose(1, 0, 2)
    F[:, 9:12, :POS - 1] = Qm[1].transpose(1, 0, 2)
    F[:, 12:15, :POS - 1] = We.transpose(1, 0, 2)
    M[:, 6:15, :POS - 1] = True
    # relative rotation at the interior Voronoi points: R[a, b] = d_a(j) . d_b(j - 1)
    R = np.einsum("akne,bkne->abne", Qm[:, :, :, 1:], Qm[:, :, :, :-1])
    F[:, 15, 1:POS - 1] = 0.5 * (R[2, 1] - R[1, 2])
    F[:, 16, 1:POS - 1] = 0.5 * (R[0, 2] - R[2, 0])
    F[:, 17, 1:POS - 1] = 0.5 * (R[1, 0] - R[0, 1])
    M[:, 15:18, 1:POS - 1] = True
    edge = np.einsum("akne,kne->ane", Qm, X[:, :, 1:] - X[:, :, :-1])
    F[:, 18:21, :POS - 1] = edge.transpose(1, 0, 2)
    M[:, 18:21, :POS - 1] = True
    F[:, 21:24, :] = np.asarray(act).T[:, :, None]
    M[:, 21:24, :] = True
    return F, M


def features(x, v, Q, w, act, in_shift, in_scale, emulate=True):
    """(nwin, 24, 51) network input: float32(raw - shift) * float32(scale), zero where a feature
    is undefined, rounded to BF16 when ``emulate``."""
    F, M = raw_features(x, v, Q, w, act)
    sh = np.asarray(in_shift, dtype=np.float64)[None, :, None]
    sc = np.asarray(in_scale, dtype=np.float64).astype(np.float32)[None, :, None]
    F32 = ((F - sh).astype(np.float32) * sc).astype(np.float64)
    F32 = np.where(M, F32, 0.0)
    return bf16(F32) if emulate else F32


def rotate_directors(Qm, w, T):
    """exp([-T w]x) applied to the director rows (Qm [3, 3, ...], w [3, ...]), by scipy's rotation
    of the rotation vector -T w."""
    from scipy.spatial.transform import Rotation
    shp = Qm.shape[2:]
    phi = (-T * w).reshape(3, -1).T
    Rm = Rotation.from_rotvec(phi).as_matrix()                  # (n, 3, 3)
    Qf = Qm.reshape(3, 3, -1).transpose(2, 0, 1)                # (n, 3 rows, 3 comps)
    out = np.einsum("nab,nbk->nak", Rm, Qf)
    return out.transpose(1, 2, 0).reshape((3, 3) + shp)


def raw_targets(s0, s1, T):
    """(nwin, 15, 51) FP64: state change over the window minus the kinematic prior (x + T v for
    positions, exp([-T w]x) Q for the directors d1, d2; none for v and w); element channels are
    zero at the last node position."""
    nwin = s0[0].shape[1] // POS
    X0, V0, Q0, W0 = _split(*s0, nwin)
    X1, V1, Q1, W1 = _split(*s1, nwin)
    D = np.zeros((nwin, N_OUT, POS))
    D[:, 0:3, :] = (X1 - X0 - T * V0).transpose(1, 0, 2)
    D[:, 3:6, :] = (V1 - V0).transpose(1, 0, 2)
    Qp = rotate_directors(Q0, W0, T)
    D[:, 6:9, :POS - 1] = (Q1[0] - Qp[0]).transpose(1, 0, 2)
    D[:, 9:12, :POS - 1] = (Q1[1] - Qp[1]).transpose(1, 0, 2)
    D[:, 12:15, :POS - 1] = (W1 - W0).transpose(1, 0, 2)
    return D


def targets(s0, s1, out_scale, T):
    """(nwin, 15, 51) training targets: float32(raw_targets / out_scale)."""
    D = raw_targets(s0, s1, T) / np.asarray(out_scale, dtype=np.float64)[None, :, None]
    return D.astype(np.float32).astype(np.float64)


def apply(state, out, out_scale, T, clamped):
    """New state from raw outputs (nwin, 51, >=15): prior + out_scale * output in FP64, directors
    by Gram-Schmidt (d1, d2; d3 = d1 x d2); clamped rods keep node 0 / element 0 at rest."""
    x, v, Q, w = [np.array(a, dtype=np.float64) for a in state]
    nwin = out.shape[0]
    X, V, Qm, We = _split(x, v, Q, w, nwin)
    o = np.asarray(out, dtype=np.float64)[:, :, :N_OUT].transpose(2, 0, 1)   # (15, nwin, 51)
    sc = np.asarray(out_scale, dtype=np.float64)[:, None, None]
    o = o * sc
    Xn = X + T * V + o[0:3]
    Vn = V + o[3:6]
    Qp = rotate_directors(Qm, We, T)
    d1 = Qp[0] + o[6:9, :, :POS - 1]
    d2 = Qp[1] + o[9:12, :, :POS - 1]
    Wn = We + o[12:15, :, :POS - 1]
    d1 = d1 / np.linalg.norm(d1, axis=0, keepdims=True)
    d2 = d2 - (d1 * d2).sum(axis=0, keepdims=True) * d1
    d2 = d2 / np.linalg.norm(d2, axis=0, keepdims=True)
    d3 = np.cross(d1, d2, axis=0)
    Qn = np.stack([d1, d2, d3])
    held = np.asarray(clamped, dtype=bool)
    Xn[:, held, 0] = X[:, held, 0]
    Vn[:, held, 0] = 0.0
    Qn[:, :, held, 0] = Qm[:, :, held, 0]
    Wn[:, held, 0] = 0.0
    return Xn.reshape(3, -1), Vn.reshape(3, -1), Qn.reshape(9, -1), Wn.reshape(3, -1)


def forward(params, F, emulate=True):
    layers = unpack(params)
    if emulate:
        layers = [(bf16(W), b.astype(np.float32).astype(np.float64)) for W, b in layers]
    feats = np.zeros((F.shape[0], 32, POS))
    feats[:, :N_FEAT] = F
    acts, pres = [feats], []
    a = feats
    for l, (W, b) in enumerate(layers):
        pre = conv(a, W, b)
        if l < 3:
            pres.append(pre)
            a = silu(pre)
            if emulate:
                a = bf16(a)
            acts.append(a)
        else:
            out = pre
    return out, (layers, acts, pres)


def loss_and_grad(params, F, T, emulate=True):
    out, (layers, acts, pres) = forward(params, F, emulate)
    r = out[:, :N_OUT, :] - T
    count = r.size
    loss = float((r * r).sum() / count)
    g = np.zeros_like(out)
    g[:, :N_OUT, :] = 2.0 * r / count
    if emulate:
        g = bf16(g)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dW, db = conv_weight_grad(g, acts[l])
        grads[l] = (dW, db)
        if l > 0:
            gin = conv_input_grad(g, W) * dsilu(pres[l - 1])
            g = bf16(gin) if emulate else gin
    return loss, pack(grads)
