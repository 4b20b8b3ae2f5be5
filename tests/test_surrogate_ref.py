"""Pins of the numpy reference of the surrogate network (CPU): its hand-derived gradient equals
central differences of its own FP64 forward loss, and its convolution equals a direct sum."""
import numpy as np

from oracle import surrogate_ref as R


def _small_batch(seed=0, nwin=2):
    rng = np.random.default_rng(seed)
    F = rng.normal(size=(nwin, R.N_FEAT, R.POS))
    T = rng.normal(size=(nwin, R.N_OUT, R.POS)) * 0.1
    params = rng.normal(size=R.n_params()) * 0.05
    return params, F, T


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 3, R.POS))
    W = rng.normal(size=(2, R.TAPS, 3))
    b = rng.normal(size=2)
    out = R.conv(x, W, b)
    for o in range(2):
        for p in (0, 1, 25, 49, 50):
            s = b[o]
            for t in range(R.TAPS):
                q = p + t - 2
                if 0 <= q < R.POS:
                    s += W[o, t] @ x[0, :, q]
            assert abs(out[0, o, p] - s) < 1e-12


def test_reference_gradient_matches_finite_differences():
    params, F, T = _small_batch()
    loss, grad = R.loss_and_grad(params, F, T, emulate=False)
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(6):
        d = rng.normal(size=params.shape)
        lp, _ = R.loss_and_grad(params + h * d, F, T, emulate=False)
        lm, _ = R.loss_and_grad(params - h * d, F, T, emulate=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad @ d) <= 1e-6 * abs(fd) + 1e-12
    # and single parameters of every layer, including biases
    offs = np.cumsum([0] + [co * R.TAPS * ci + co for co, ci in R.SHAPES])
    for l in range(4):
        for k in (offs[l] + 3, offs[l + 1] - 1):
            e = np.zeros_like(params)
            e[k] = 1.0
            lp, _ = R.loss_and_grad(params + h * e, F, T, emulate=False)
            lm, _ = R.loss_and_grad(params - h * e, F, T, emulate=False)
            assert abs((lp - lm) / (2 * h) - grad[k]) <= 1e-6 * max(abs(grad[k]), 1e-8)


def test_bf16_rounding_is_round_to_nearest_even():
    # BF16 keeps 7 fraction bits: the ulp at 1 is 2^-7, so 1 + 2^-8 is an exact tie
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 1.0 + 3 * 2 ** -8, -2.5, 0.0])
    got = R.bf16(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0                     # tie rounds to the even neighbour 1.0
    assert got[2] == 1.0                     # below the half ulp rounds down
    assert got[3] == 1.0 + 2 ** -7           # above the half ulp rounds up
    assert got[4] == 1.0 + 2 ** -6           # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert got[5] == -2.5 and got[6] == 0.0


# ---- features, targets and the state update, pinned to closed forms and to the oracle's step

def _straight_rods(nwin, rng=None, l=0.004):
    """nwin straight rods of 50 elements, each along the third director of a random rotation."""
    from scipy.spatial.transform import Rotation
    rng = rng or np.random.default_rng(0)
    x = np.zeros((3, nwin * R.POS))
    Q = np.zeros((9, nwin * (R.POS - 1)))
    for b in range(nwin):
        Rm = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()   # columns d1, d2, d3
        base = rng.normal(size=3)
        for j in range(R.POS):
            x[:, b * R.POS + j] = base + j * l * Rm[:, 2]
        for j in range(R.POS - 1):
            Q[:, b * (R.POS - 1) + j] = Rm.T.reshape(-1)                              # rows are directors
    return x, np.zeros_like(x), Q, np.zeros((3, Q.shape[1]))


def test_edge_feature_of_a_straight_rod_is_the_rest_edge_in_any_orientation():
    l = 0.004
    x, v, Q, w = _straight_rods(4, l=l)
    F, M = R.raw_features(x, v, Q, w, np.zeros((3, 4)))
    assert np.allclose(F[:, 18, :50], 0.0, atol=1e-15) and np.allclose(F[:, 19, :50], 0.0, atol=1e-15)
    assert np.allclose(F[:, 20, :50], l, rtol=1e-12)
    assert not M[:, 18:21, 50].any() and M[:, 18:21, :50].all()
    # no relative rotation along a straight rod; undefined at both ends
    assert np.abs(F[:, 15:18]).max() < 1e-15
    assert not M[:, 15:18, 0].any() and not M[:, 15:18, 50].any() and M[:, 15:18, 1:50].all()
    # positions relative to the base node, velocities as given
    assert np.allclose(F[:, 0:3, 0], 0.0) and np.allclose(np.linalg.norm(F[:, 0:3, 50], axis=1), 50 * l)


def test_rotation_feature_of_an_arc_is_minus_sine_of_the_turn():
    """Element j turned by j*alpha about the lab x axis: R = Q_j Q_{j-1}^T is a turn by -alpha
    about d1, so the feature is (-sin alpha, 0, 0)."""
    from scipy.spatial.transform import Rotation
    alpha = 0.013
    nwin = 1
    Q = np.zeros((9, 50))
    x = np.zeros((3, 51))
    for j in range(50):
        Rm = Rotation.from_rotvec([j * alpha, 0.0, 0.0]).as_matrix()
        Q[:, j] = Rm.T.reshape(-1)
        x[:, j + 1] = x[:, j] + 0.004 * Rm[:, 2]
    F, _ = R.raw_features(x, np.zeros_like(x), Q, np.zeros((3, 50)), np.zeros((3, nwin)))
    assert np.allclose(F[0, 15, 1:50], -np.sin(alpha), rtol=1e-12)
    assert np.abs(F[0, 16:18, 1:50]).max() < 1e-15
    assert np.allclose(F[0, 20, :50], 0.004, rtol=1e-12)     # each edge is along its own d3


def test_targets_vanish_for_a_rigid_motion_stepped_by_the_oracle():
    """A free, force-free straight rod translating with uniform v and spinning about its own
    axis (a principal axis) moves rigidly: after one window of the oracle's steps the state is
    the kinematic prior exactly, so every target is zero up to rounding; the prior with zero
    network output reproduces the oracle's state."""
    import rodgen
    from oracle.oracle import Oracle
    p = rodgen.cilia_carpet(side=1, n=50, gamma=0.0)
    p = p.replace(act_amp=None, act_period=None, act_phase=None, clamp_base=np.zeros(1, dtype=np.int8))
    x, v, Q, w = p.state()
    v[:] = np.array([0.3, -0.2, 0.1])[:, None]
    w[:] = np.array([0.0, 0.0, 7.0])[:, None]             # about d3, the rod's axis
    dt, W = 1e-5, 50
    s1 = Oracle(p).step(x, v, Q, w, dt=dt, n_steps=W)
    D = R.raw_targets((x, v, Q, w), s1, W * dt)
    assert np.abs(D[:, 0:3]).max() < 1e-14                 # positions: x + T v
    assert np.abs(D[:, 3:6]).max() < 1e-10                 # velocities unchanged (rounding-level forces)
    assert np.abs(D[:, 6:12]).max() < 1e-12                # directors: exp([-T w]x) Q
    assert np.abs(D[:, 12:15]).max() < 1e-10               # angular velocity unchanged
    # a sign error in the prior's rotation would leave 2 sin(T |w|) ~ 7e-3 in the director channels
    xn, vn, Qn, wn = R.apply((x, v, Q, w), np.zeros((1, 51, 16)), np.ones(15), W * dt, [False])
    assert np.abs(xn - s1[0]).max() < 1e-14 and np.abs(Qn - s1[2]).max() < 1e-12


def test_apply_keeps_directors_orthonormal_and_the_clamp():
    rng = np.random.default_rng(4)
    x, v, Q, w = _straight_rods(3, rng)
    v = rng.normal(size=v.shape) * 0.1
    w = rng.normal(size=w.shape)
    out = rng.normal(size=(3, 51, 16)) * 0.5
    scale = np.full(15, 1e-3)
    xn, vn, Qn, wn = R.apply((x, v, Q, w), out, scale, 5e-4, [True, False, True])
    Qm = Qn.reshape(3, 3, -1)
    G = np.einsum("ake,bke->abe", Qm, Qm)
    assert np.abs(G - np.eye(3)[:, :, None]).max() < 1e-14
    assert np.all(np.linalg.det(Qm.transpose(2, 0, 1)) > 0)
    for b, held in enumerate([True, False, True]):
        n0, e0 = b * 51, b * 50
        if held:
            assert np.array_equal(xn[:, n0], x[:, n0]) and not vn[:, n0].any()
            assert np.array_equal(Qn[:, e0], Q[:, e0]) and not wn[:, e0].any()
        else:
            assert not np.array_equal(xn[:, n0], x[:, n0])
    # free entries: x = x + T v + scale * out exactly
    b, j = 1, 7
    assert np.allclose(xn[:, b * 51 + j], x[:, b * 51 + j] + 5e-4 * v[:, b * 51 + j] + 1e-3 * out[b, j, 0:3],
                       rtol=0, atol=1e-16)
