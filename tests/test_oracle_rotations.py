"""Oracle pins: rotation exponential / logarithm and the director update direction.

The rotation vector convention is fixed by the model: omega = ax(Q dQ^T/dt) with the rows of
Q the directors (Methods), so the exact flow for constant omega is Q(t+h) = exp(-h[omega]x) Q(t);
the exponential and logarithm themselves are pinned against scipy's Rotation (a library
routine with the same active-rotation convention, R = exp([phi]x)).
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle, rot_exp, rot_log

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def _random_rotvecs(rng, n, max_angle):
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.uniform(0.0, max_angle, n)
    return axis * ang[:, None]


def test_exp_matches_scipy():
    rng = np.random.default_rng(0)
    phis = np.concatenate([_random_rotvecs(rng, 200, np.pi - 1e-3),
                           _random_rotvecs(rng, 50, 1e-6), _random_rotvecs(rng, 50, 1e-10)])
    for phi in phis:
        R = rot_exp(phi)
        assert np.abs(R - Rotation.from_rotvec(phi).as_matrix()).max() < 4e-16 * 8
    assert np.array_equal(rot_exp(np.zeros(3)), np.eye(3))


def test_log_matches_scipy():
    rng = np.random.default_rng(1)
    phis = np.concatenate([_random_rotvecs(rng, 200, np.pi - 1e-3), _random_rotvecs(rng, 50, 1e-5)])
    for phi in phis:
        R = Rotation.from_rotvec(phi).as_matrix()
        got = rot_log(R)
        ref = Rotation.from_matrix(R).as_rotvec()
        assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.linalg.norm(ref)) * 10


def test_log_exp_roundtrip_small_angles():
    rng = np.random.default_rng(2)
    for scale in (1e-12, 1e-8, 1e-4, 1e-2, 1.0):
        phi = rng.normal(size=3) * scale
        back = rot_log(rot_exp(phi))
        assert np.abs(back - phi).max() <= 1e-15 * max(np.linalg.norm(phi), 1e-300) * 10 + 1e-30


def test_director_update_direction_for_spin_about_d3():
    """A single free element spinning with local omega = (0, 0, w): after one step of h the
    body has turned by +w h about d3 (lab angular velocity w d3, right-hand rule), so
    d1(t+h) = cos(wh) d1 + sin(wh) d2 and d3 is unchanged."""
    p = rodgen.cantilever(n=1, length=0.01, tip_force=0.0, nu=0.0)
    p = p.replace(clamp_base=None, tip_force=None)
    wz, h = 3.0, 1e-3
    x, v, Q, w = p.state()
    w[:, 0] = [0.0, 0.0, wz]
    o = Oracle(p)
    x1, v1, Q1, w1 = o.step(x, v, Q, w, h, 1)
    d1, d2, d3 = Q[0:3, 0], Q[3:6, 0], Q[6:9, 0]
    c, s = np.cos(wz * h), np.sin(wz * h)
    assert np.abs(Q1[0:3, 0] - (c * d1 + s * d2)).max() < 1e-15
    assert np.abs(Q1[3:6, 0] - (-s * d1 + c * d2)).max() < 1e-15
    assert np.abs(Q1[6:9, 0] - d3).max() < 1e-15
    assert np.abs(w1[:, 0] - [0.0, 0.0, wz]).max() < 1e-15


def test_directors_stay_orthonormal():
    """Proper orthogonality of Q (Methods) survives 10^4 steps of a driven, damped rod."""
    p = rodgen.perturbed(rodgen.cantilever(n=20, length=0.2, tip_force=1e-3), seed=3, rot=0.1, omega=20.0)
    o = Oracle(p)
    x, v, Q, w = o.step(*p.state(), dt=1e-5, n_steps=10_000)
    assert o.orthonormality_error(Q) < 1e-12
    for i in range(Q.shape[1]):
        assert np.linalg.det(Q[:, i].reshape(3, 3)) > 0
