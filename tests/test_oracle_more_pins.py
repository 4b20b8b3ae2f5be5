"""More oracle pins: conservation of angular momentum, closed-form dynamics and load laws.

* angular momentum of a free, unloaded rod, L = sum x_j x m_j v_j + sum Q_i^T (J_i/e_i) w_i
  (J/e: the inertia per current length that Eq. 1b's left side carries), is conserved: the
  transport terms (J w/e) x w and (J w/e^2) de/dt of Eq. 1b are exactly what makes d/dt of the
  spin part equal Q^T (tau_bend + tau_shear), and the shear couple balances the orbital part;
* the lowest axial mode of a clamped-free rod has period 4 L / sqrt(E/rho) (wave equation limit
  of Eq. 1a, lumped masses);
* linear damping decays translation and rotation at the same rate nu/(rho A); Stokes drag
  decays translation at gamma/(rho A) and leaves rotation alone;
* free fall: every node follows x0 + g t^2/2 (Verlet is exact for constant acceleration);
* a stretched arc with rest stretch sigma0 = (0, 0, e-1) carries the couple B kappa / e^3
  (the 1/e^3 of Eq. 1b's bending term);
* the base actuation couple A sin(phi) about d1, held constant (T -> infinity), is balanced
  by the bend at the clamp: kappa_0 = A / EI.
"""
import numpy as np

import rodgen
from oracle.oracle import Oracle


def _free_rod(n=20, length=0.2, radius=0.01):
    return rodgen.cantilever(n=n, length=length, radius=radius, tip_force=0.0, nu=0.0).replace(
        clamp_base=None, tip_force=None)


def _angular_momentum(p, x, v, Q, w, o):
    r = p.radius[0]
    A = np.pi * r * r
    I = np.pi * r ** 4 / 4
    Ivec = np.array([I, I, 2 * I])
    rl = p.rest_len
    m = np.zeros(p.n_nodes)
    m[:-1] += 0.5 * 1000 * A * rl
    m[1:] += 0.5 * 1000 * A * rl
    _, _, dil, _ = o.strains(x, Q)
    L = np.cross(x.T, (m * v).T).sum(0)
    for i in range(p.n_elems):
        Jw = 1000 * rl[i] * Ivec * w[:, i] / dil[i]
        L += Q[:, i].reshape(3, 3).T @ Jw
    return L


def _momentum_drift(dt, T=0.02):
    p = rodgen.perturbed(_free_rod(), seed=21, pos=0.01, vel=0.2, rot=0.02, omega=30.0)
    x, v, Q, w = p.state()
    # add a stretching velocity field so that de/dt is far from zero
    v[2] += 40.0 * (x[2] - x[2].mean())
    o = Oracle(p)
    L0 = _angular_momentum(p, x, v, Q, w, o)
    st = (x, v, Q, w)
    worst = 0.0
    n = int(round(T / dt))
    for _ in range(10):
        st = o.step(*st, dt=dt, n_steps=n // 10)
        worst = max(worst, np.abs(_angular_momentum(p, *st, o) - L0).max())
    return worst / np.abs(L0).max()


def test_angular_momentum_conserved():
    """Conserved up to a first-order time-stepping error that vanishes as dt -> 0."""
    e1 = _momentum_drift(1e-5)
    e2 = _momentum_drift(5e-6)
    assert e2 < 1.5e-4
    assert 1.5 < e1 / e2 < 3.0


def test_axial_mode_period():
    n, L = 40, 0.5
    p = rodgen.cantilever(n=n, length=L, radius=0.01, tip_force=0.0, nu=0.0, dt=2e-6)
    x, v, Q, w = p.state()
    x = x.copy()
    x[2] *= 1.0 + 1e-4           # small uniform stretch, released at rest
    o = Oracle(p)
    dt, steps = 2e-6, 40
    tip = []
    st = (x, v, Q, w)
    for _ in range(1000):
        st = o.step(*st, dt=dt, n_steps=steps)
        tip.append(st[0][2, -1] - L)
    tip = np.array(tip)
    t = (np.arange(1, len(tip) + 1)) * dt * steps
    # downward zero crossings of the tip displacement about its mean
    s = tip - tip.mean()
    idx = np.where((s[:-1] > 0) & (s[1:] <= 0))[0]
    tc = t[idx] - s[idx] * (t[idx + 1] - t[idx]) / (s[idx + 1] - s[idx])
    period = np.diff(tc).mean()
    expect = 4 * L / np.sqrt(1e6 / 1000.0)
    assert abs(period / expect - 1) < 5e-3


def test_damping_and_drag_rates():
    nu, gamma = 0.3, 0.2
    r = 0.01
    rhoA = 1000 * np.pi * r * r
    p = _free_rod().replace(nu_damp=nu)
    x, v, Q, w = p.state()
    v[0] = 0.5
    w[2] = 7.0
    T, dt = 0.05, 1e-5
    x1, v1, Q1, w1 = Oracle(p).step(x, v, Q, w, dt=dt, n_steps=int(T / dt))
    decay = np.exp(-nu / rhoA * T)
    assert np.abs(v1[0] / 0.5 - decay).max() < 1e-3
    assert np.abs(w1[2] / 7.0 - decay).max() < 1e-3
    q = _free_rod().replace(stokes_gamma=gamma)
    x1, v1, Q1, w1 = Oracle(q).step(x, v, Q, w, dt=dt, n_steps=int(T / dt))
    assert np.abs(v1[0] / 0.5 - np.exp(-gamma / rhoA * T)).max() < 1e-3
    assert np.abs(w1[2] - 7.0).max() < 1e-9


def test_free_fall():
    g = np.array([0.3, -2.0, -9.81])
    p = _free_rod().replace(gravity=g)
    x, v, Q, w = p.state()
    T, dt = 0.01, 1e-4
    x1, v1, Q1, w1 = Oracle(p).step(x, v, Q, w, dt=dt, n_steps=100)
    # strain round-off (rest lengths are not binary fractions) gives ~1e-12 m/s of noise
    assert np.abs(x1 - (x + 0.5 * g[:, None] * T * T)).max() < 1e-13
    assert np.abs(v1 - g[:, None] * T).max() < 1e-10


def test_stretched_arc_couple_scales_with_inverse_cube_stretch():
    n, L, r, e = 30, 1.0, 0.01, 1.1
    I = np.pi * r ** 4 / 4
    EI = 1e6 * I
    kappa = 0.02
    dtheta = kappa * L / n
    th = (np.arange(n) + 0.5) * dtheta
    d1 = np.stack([np.ones(n), np.zeros(n), np.zeros(n)])
    d2 = np.stack([np.zeros(n), np.cos(th), np.sin(th)])
    d3 = np.stack([np.zeros(n), -np.sin(th), np.cos(th)])
    Q = np.concatenate([d1, d2, d3])
    x = np.concatenate([np.zeros((3, 1)), np.cumsum(e * (L / n) * d3, axis=1)], axis=1)
    rest_sigma = np.zeros((3, n))
    rest_sigma[2] = e - 1.0
    M = EI * kappa / e ** 3
    couple = np.zeros((3, n))
    couple[0, -1] = M
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=0.0, nu=0.0).replace(
        tip_force=None, rest_sigma=rest_sigma, elem_couple=couple)
    av, aw = Oracle(p).rhs(x, np.zeros_like(x), Q, np.zeros((3, n)))
    J = 1000 * (L / n) * I
    assert np.abs(aw).max() * J / M < 1e-8


def test_base_actuation_couple_static_balance():
    n, L, r = 20, 0.2, 0.005
    I = np.pi * r ** 4 / 4
    EI = 1e6 * I
    A0 = 2e-5
    dtheta = A0 / EI * (L / n)       # kappa_0 = A0/EI over the Voronoi length L/n
    th = np.where(np.arange(n) >= 1, dtheta, 0.0)
    d1 = np.stack([np.ones(n), np.zeros(n), np.zeros(n)])
    d2 = np.stack([np.zeros(n), np.cos(th), np.sin(th)])
    d3 = np.stack([np.zeros(n), -np.sin(th), np.cos(th)])
    Q = np.concatenate([d1, d2, d3])
    x = np.concatenate([np.zeros((3, 1)), np.cumsum((L / n) * d3, axis=1)], axis=1)
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=0.0, nu=0.0).replace(
        tip_force=None, act_amp=np.array([A0]), act_period=np.array([1e12]), act_phase=np.array([np.pi / 2]))
    av, aw = Oracle(p).rhs(x, np.zeros_like(x), Q, np.zeros((3, n)), t=0.0)
    J = 1000 * (L / n) * I
    assert np.abs(aw).max() * J / A0 < 1e-8
    # the opposite phase is not balanced
    q = p.replace(act_phase=np.array([-np.pi / 2]))
    av, aw = Oracle(q).rhs(x, np.zeros_like(x), Q, np.zeros((3, n)), t=0.0)
    assert np.abs(aw[0, 1]) * J / A0 > 1.0
