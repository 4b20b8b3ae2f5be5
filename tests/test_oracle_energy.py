"""Oracle pins for the rod's energy (the quantity the GPU diagnostics reproduce).

Closed forms of the Cosserat rod (Methods: the model behind Eq. 1) on one rod of length L with
non-uniform rest lengths (so that a Voronoi length D_k = (rl_k + rl_{k+1}) / 2 differs from
the element lengths around it), circular section A = pi r^2, I_1 = I_2 = pi r^4 / 4,
I_3 = 2 I_1:
  * rigid translation V:          1/2 rho A L |V|^2
  * uniform angular velocity W:   1/2 rho L (I_1 W_1^2 + I_2 W_2^2 + I_3 W_3^2)
  * uniform shear and stretch, sigma = (g1, g2, s):  1/2 L (alpha G A (g1^2 + g2^2) + E A s^2)
  * uniform bending kappa_0 about d1, an arc whose relative rotations are kappa_0 D_k:
                                   1/2 E I_1 kappa_0^2 sum_k D_k = 1/2 E I_1 kappa_0^2 (L - rl_0/2 - rl_{n-1}/2)
  * uniform twist tau:             1/2 G I_3 tau^2 (L - rl_0/2 - rl_{n-1}/2)
  * gravity on a rod along z from 0 to L: -rho A g_z L^2 / 2 (the node masses integrate a linear
    function exactly); a tip force F: -F . x_tip
and the sum of all of them at once (the parts are independent).
"""
import numpy as np

import rodgen
from oracle.oracle import Oracle

R, E_MOD, G_MOD, RHO, ALPHA = 0.01, 1e6, 1e6 / 1.5, 1000.0, 4.0 / 3.0
A = np.pi * R ** 2
I1 = np.pi * R ** 4 / 4


def _rod(n=40, L=1.0, seed=0):
    """Straight rod along lab z with frames d1 = x, d2 = y, d3 = z and rest lengths that vary by
    +-50 % about L/n (normalised to total L)."""
    rng = np.random.default_rng(seed)
    rl = rng.uniform(0.5, 1.5, n)
    rl *= L / rl.sum()
    p = rodgen.cantilever(n=n, length=L, radius=R, youngs=E_MOD, tip_force=0.0, nu=0.0, density=RHO)
    z = np.concatenate([[0.0], np.cumsum(rl)])
    x = np.zeros((3, n + 1))
    x[2] = z
    return p.replace(rest_len=rl, x=x, clamp_base=None, tip_force=None, alpha_c=ALPHA)


def _H(p):
    return Oracle(p).energy(*p.state())


def _rot_x(phi):
    c, s = np.cos(phi), np.sin(phi)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _frames_to_Q(d1, d2, d3):
    return np.concatenate([d1, d2, d3], axis=0)   # rows d1 (3, n), d2, d3 -> (9, n)


def test_rigid_translation():
    p = _rod()
    V = np.array([0.3, -1.2, 0.7])
    p = p.replace(v=np.tile(V[:, None], (1, p.n_nodes)))
    L = p.rest_len.sum()
    assert np.isclose(_H(p), 0.5 * RHO * A * L * V @ V, rtol=1e-12, atol=0)


def test_uniform_angular_velocity():
    p = _rod()
    W = np.array([2.0, -3.0, 5.0])
    p = p.replace(w=np.tile(W[:, None], (1, p.n_elems)))
    L = p.rest_len.sum()
    ref = 0.5 * RHO * L * (I1 * W[0] ** 2 + I1 * W[1] ** 2 + 2 * I1 * W[2] ** 2)
    assert np.isclose(_H(p), ref, rtol=1e-12, atol=0)


def test_uniform_shear_and_stretch():
    p = _rod()
    g1, g2, s = 0.02, -0.015, 0.03
    l_dir = np.array([g1, g2, 1.0 + s])
    x = np.concatenate([np.zeros((3, 1)), np.cumsum(l_dir[:, None] * p.rest_len[None, :], axis=1)], axis=1)
    p = p.replace(x=x)
    L = p.rest_len.sum()
    ref = 0.5 * L * (ALPHA * G_MOD * A * (g1 ** 2 + g2 ** 2) + E_MOD * A * s ** 2)
    assert np.isclose(_H(p), ref, rtol=1e-11, atol=0)


def _arc(p, kappa0):
    """Frames turned about lab x by kappa0 * D_k from element to element, nodes following the
    chords: sigma = 0 and kappa = kappa0 about d1 at every Voronoi point."""
    rl = p.rest_len
    D = 0.5 * (rl[:-1] + rl[1:])
    phi = np.concatenate([[0.0], np.cumsum(kappa0 * D)])
    d1 = np.tile(np.array([[1.0], [0.0], [0.0]]), (1, rl.size))
    d3 = np.stack([_rot_x(f) @ np.array([0.0, 0.0, 1.0]) for f in phi], axis=1)
    d2 = np.cross(d3.T, d1.T).T
    x = np.concatenate([np.zeros((3, 1)), np.cumsum(d3 * rl[None, :], axis=1)], axis=1)
    return p.replace(x=x, Q=_frames_to_Q(d1, d2, d3)), D.sum()


def test_uniform_bending():
    p = _rod()
    kappa0 = 2.5
    q, sumD = _arc(p, kappa0)
    L = p.rest_len.sum()
    assert np.isclose(sumD, L - p.rest_len[0] / 2 - p.rest_len[-1] / 2)
    assert np.isclose(_H(q), 0.5 * E_MOD * I1 * kappa0 ** 2 * sumD, rtol=1e-11, atol=0)


def test_uniform_twist():
    p = _rod()
    tau = 4.0
    rl = p.rest_len
    D = 0.5 * (rl[:-1] + rl[1:])
    psi = np.concatenate([[0.0], np.cumsum(tau * D)])
    c, s = np.cos(psi), np.sin(psi)
    d1 = np.stack([c, s, np.zeros_like(c)])
    d2 = np.stack([-s, c, np.zeros_like(c)])
    d3 = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, rl.size))
    q = p.replace(Q=_frames_to_Q(d1, d2, d3))
    assert np.isclose(_H(q), 0.5 * G_MOD * 2 * I1 * tau ** 2 * D.sum(), rtol=1e-11, atol=0)


def test_gravity_and_tip_force_potential():
    p = _rod()
    L = p.rest_len.sum()
    g = np.array([0.0, 0.0, -9.81])
    F = np.array([0.1, -0.2, 0.3])
    q = p.replace(gravity=g, tip_force=F[:, None])
    ref = -RHO * A * g[2] * L ** 2 / 2 - F @ np.array([0.0, 0.0, L])
    assert np.isclose(_H(q), ref, rtol=1e-12, atol=0)


def test_parts_add_up():
    p = _rod()
    kappa0 = 1.5
    q, sumD = _arc(p, kappa0)
    V = np.array([0.1, 0.2, -0.1])
    W = np.array([1.0, 0.5, -2.0])
    q = q.replace(v=np.tile(V[:, None], (1, q.n_nodes)), w=np.tile(W[:, None], (1, q.n_elems)))
    L = p.rest_len.sum()
    ref = (0.5 * RHO * A * L * V @ V + 0.5 * RHO * L * I1 * (W[0] ** 2 + W[1] ** 2 + 2 * W[2] ** 2)
           + 0.5 * E_MOD * I1 * kappa0 ** 2 * sumD)
    assert np.isclose(_H(q), ref, rtol=1e-11, atol=0)
