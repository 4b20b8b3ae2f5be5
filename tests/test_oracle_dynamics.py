"""Oracle pins from dynamics and conservation laws.

* rigid translation: no internal load, x(t) = x0 + v t (Eq. 1a with zero strain);
* torque-free spin of a straight rod about its axis: omega and the straight shape persist
  (Eq. 1b: (J w / e) x w = 0 for w along a principal axis, no curvature is created);
* linear momentum of a free, unloaded rod is conserved exactly (the difference operator
  telescopes);
* the discrete Kirchhoff helix: uniform kappa = (k1, 0, k3) with the wrench n = -k3 (EI - GJ) kappa
  balances kappa x B kappa + e3 x n = 0 (Eq. 1b, steady uniform state), so interior elements and
  nodes carry no load;
* undamped energy: no secular drift; the energy error of the scheme scales with the strain
  amplitude (the 1/e and 1/eps^3 factors make the forces the gradient of the quadratic energy
  only at first order), and it is small at small strain.
"""
import numpy as np

import rodgen
from oracle.oracle import Oracle, rot_exp


def _free_rod(n=20, length=0.2, radius=0.01):
    return rodgen.cantilever(n=n, length=length, radius=radius, tip_force=0.0, nu=0.0).replace(
        clamp_base=None, tip_force=None)


def test_rigid_translation():
    p = _free_rod()
    x, v, Q, w = p.state()
    v[:] = np.array([0.3, -1.2, 0.7])[:, None]
    o = Oracle(p)
    x1, v1, Q1, w1 = o.step(x, v, Q, w, dt=1e-4, n_steps=100)
    assert np.abs(v1 - v).max() < 1e-12
    assert np.abs(x1 - (x + v * 1e-2)).max() < 1e-13
    assert np.abs(Q1 - Q).max() == 0.0


def test_torque_free_spin_about_axis():
    p = _free_rod()
    x, v, Q, w = p.state()
    w[2] = 40.0
    o = Oracle(p)
    x1, v1, Q1, w1 = o.step(x, v, Q, w, dt=1e-5, n_steps=500)
    assert np.abs(w1 - w).max() < 1e-10
    assert np.abs(x1 - x).max() < 1e-15
    _, kap, _, _ = o.strains(x1, Q1)
    assert np.abs(kap).max() < 1e-9
    ang = 40.0 * 500 * 1e-5
    d1 = Q[0:3, 0]
    d2 = Q[3:6, 0]
    assert np.abs(Q1[0:3, 5] - (np.cos(ang) * d1 + np.sin(ang) * d2)).max() < 1e-12


def test_linear_momentum_conserved_for_free_rod():
    p = rodgen.perturbed(_free_rod(), seed=4, pos=0.02, vel=0.3, rot=0.1, omega=10.0)
    o = Oracle(p)
    m = np.full(p.n_nodes, 1000 * np.pi * 0.01 ** 2 * 0.2 / 20)
    m[0] *= 0.5
    m[-1] *= 0.5
    P0 = (p.v * m).sum(1)
    x, v, Q, w = o.step(*p.state(), dt=1e-5, n_steps=2000)
    P1 = (v * m).sum(1)
    assert np.abs(P1 - P0).max() < 1e-12


def test_kirchhoff_helix_is_balanced():
    n, L, r = 30, 0.3, 0.01
    p = _free_rod(n=n, length=L, radius=r)
    E, G = 1e6, 1e6 / 1.5
    A = np.pi * r * r
    I = np.pi * r ** 4 / 4
    EI, GJ = E * I, G * 2 * I
    S = np.array([4 / 3 * G * A, 4 / 3 * G * A, E * A])
    kappa = np.array([2.0, 0.0, 3.0])
    nvec = -kappa[2] * (EI - GJ) * kappa
    sigma = nvec / S
    rl = L / n
    # frames: Q_{k+1} = exp(-rl [kappa]x) Q_k  (rotation about the body-fixed axis kappa)
    Rstep = rot_exp(-rl * kappa)
    Qs = [np.eye(3)]
    for _ in range(n - 1):
        Qs.append(Rstep @ Qs[-1])
    x = np.zeros((3, n + 1))
    for i in range(n):
        x[:, i + 1] = x[:, i] + rl * Qs[i].T @ (sigma + np.array([0, 0, 1.0]))
    Q = np.stack([q.reshape(9) for q in Qs], axis=1)
    o = Oracle(p)
    _, kap, dil, _ = o.strains(x, Q)
    assert np.abs(kap - kappa[:, None]).max() < 1e-10
    av, aw = o.rhs(x, np.zeros_like(x), Q, np.zeros((3, n)))
    J = 1000 * rl * I
    m = 1000 * A * rl
    T = np.abs(np.cross(kappa, [EI, EI, GJ] * kappa)).max() * rl     # magnitude of one averaged term
    # interior elements / nodes balanced to the strain order of the 1/e, 1/eps^3 factors
    assert np.abs(aw[:, 1:-1]).max() * J < 1e-3 * T
    assert np.abs(av[:, 2:-2]).max() * m < 1e-9 * np.abs(nvec).max() + 1e-14
    # without the shear wrench the same helix is not balanced
    x0 = np.zeros((3, n + 1))
    for i in range(n):
        x0[:, i + 1] = x0[:, i] + rl * Qs[i].T @ np.array([0, 0, 1.0])
    av, aw = o.rhs(x0, np.zeros_like(x0), Q, np.zeros((3, n)))
    assert np.abs(aw[:, 1:-1]).max() * J > 0.5 * T


def _energy_run(amp, dt, steps=8000, chunks=40):
    p = rodgen.perturbed(_free_rod(), seed=5, pos=0.02 * amp, vel=0.0, rot=0.05 * amp, omega=0.0)
    o = Oracle(p)
    st = p.state()
    H0 = o.energy(*st)
    Hs = []
    for _ in range(chunks):
        st = o.step(*st, dt=dt, n_steps=steps // chunks)
        Hs.append(o.energy(*st))
    Hs = np.array(Hs)
    return np.abs(Hs - H0).max() / H0, (Hs[-10:].mean() - Hs[:10].mean()) / H0


def test_undamped_energy_error_is_small_and_scales_with_strain():
    # small strain: the error is the bounded O(dt^2)-type oscillation of the symplectic scheme
    e1, d1 = _energy_run(0.01, 1e-5)
    e4, d4 = _energy_run(0.01, 2.5e-6, steps=32000)
    assert e4 < 2e-4 and abs(d4) < 2e-4
    assert e1 > 2.0 * e4
    # larger strain: a dt-independent error that grows with the strain amplitude
    e_mid, _ = _energy_run(0.1, 1e-5)
    e_big, _ = _energy_run(1.0, 1e-5)
    e_big_half, _ = _energy_run(1.0, 5e-6, steps=16000)
    assert abs(e_big_half / e_big - 1) < 0.25
    assert 5.0 < e_big / e_mid < 50.0
    assert e_big < 0.05
