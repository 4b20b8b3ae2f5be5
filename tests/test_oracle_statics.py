"""Oracle pins from statics: configurations whose equilibrium the continuum model fixes.

* zero internal load at the rest configuration (Eq. 1 with sigma = sigma0, kappa = kappa0);
* uniform stretch of a clamped rod under an axial end force F: equilibrium of Eq. 1a needs
  Q^T S sigma / e = F everywhere, i.e. EA (e - 1)/e = F, e = 1/(1 - F/EA);
* uniform bending under an end couple M about d1: Eq. 1b needs B kappa = M, kappa = M/EI,
  a circular arc bending away from +y for M > 0 (right-hand rule);
* the static cantilever: tip deflection F L^3/(3EI) + F L/(alpha_c G A) (Timoshenko beam with
  the model's shear stiffness alpha_c G A), approached at first order in the element length.
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle


def _consts(r, E=1e6, G=1e6 / 1.5, alpha=4 / 3):
    A = np.pi * r * r
    I = np.pi * r ** 4 / 4
    return A, I, E * A, E * I, alpha * G * A


def test_straight_rod_at_rest_has_zero_rhs():
    p = rodgen.cantilever(n=30, tip_force=0.0, nu=0.0).replace(clamp_base=None, tip_force=None)
    av, aw = Oracle(p).rhs(*p.state())
    assert np.abs(av).max() < 1e-9 and np.abs(aw).max() < 1e-9


def test_any_shape_with_its_own_rest_strains_is_unloaded():
    base = rodgen.cantilever(n=25, tip_force=0.0, nu=0.0).replace(clamp_base=None, tip_force=None)
    p = rodgen.perturbed(base, seed=11, pos=0.05, vel=0.0, rot=0.3, omega=0.0)
    o = Oracle(p)
    x, v, Q, w = p.state()
    sig, kap, _, _ = o.strains(x, Q)
    q = p.replace(rest_sigma=sig, rest_kappa=kap)
    av, aw = Oracle(q).rhs(x, v, Q, w)
    # scale: forces S*|sigma| ~ 1e2 N on masses ~1e-3 kg -> 1e5; compare against that
    assert np.abs(av).max() < 1e-6 and np.abs(aw).max() < 1e-4
    # and the same shape without rest strains is loaded
    av2, aw2 = Oracle(p).rhs(x, v, Q, w)
    assert np.abs(av2).max() > 1.0


@pytest.mark.parametrize("F", [5.0, -12.0, 20.0])
def test_uniform_stretch_closed_form(F):
    n, L, r = 20, 1.0, 0.01
    A, I, EA, EI, GAs = _consts(r)
    e = 1.0 / (1.0 - F / EA)
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=0.0, nu=0.0)
    p = p.replace(tip_force=np.array([[0.0], [0.0], [F]]))
    x, v, Q, w = p.state()
    x = x.copy()
    x[2] = np.arange(n + 1) * (L / n) * e
    av, aw = Oracle(p).rhs(x, v, Q, w)
    m_node = 1000 * A * L / n
    # residual force relative to F
    assert np.abs(av).max() * m_node / abs(F) < 1e-9
    assert np.abs(aw).max() < 1e-9
    # a wrong law (linear e = 1 + F/EA) leaves a clearly nonzero tip residual
    x[2] = np.arange(n + 1) * (L / n) * (1 + F / EA)
    av, aw = Oracle(p).rhs(x, v, Q, w)
    assert np.abs(av[2, -1]) * 0.5 * m_node / abs(F) > 1e-3


def _arc_state(n, L, dtheta):
    """Nodes on a circle bending toward -y in the y-z plane; element chords of length L/n and
    directors d1 = x, d3 = chord direction (rotation of the straight frame about +x)."""
    rl = L / n
    th = (np.arange(n) + 0.5) * dtheta
    d1 = np.stack([np.ones(n), np.zeros(n), np.zeros(n)])
    d2 = np.stack([np.zeros(n), np.cos(th), np.sin(th)])
    d3 = np.stack([np.zeros(n), -np.sin(th), np.cos(th)])
    Q = np.concatenate([d1, d2, d3])
    # consecutive chords of length rl along d3 put the nodes on the circle of radius
    # rl / (2 sin(dtheta/2)) without the cancellation of R (cos - 1)
    x = np.concatenate([np.zeros((3, 1)), np.cumsum(rl * d3, axis=1)], axis=1)
    return x, Q


@pytest.mark.parametrize("M", [1e-4, 5e-4])
def test_uniform_bending_closed_form(M):
    n, L, r = 40, 1.0, 0.01
    A, I, EA, EI, GAs = _consts(r)
    kappa = M / EI
    dtheta = kappa * L / n
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=0.0, nu=0.0).replace(tip_force=None)
    x, Q = _arc_state(n, L, dtheta)
    couple = np.zeros((3, n))
    couple[0, -1] = M
    q = p.replace(elem_couple=couple)
    o = Oracle(q)
    sig, kap, _, _ = o.strains(x, Q)
    assert np.abs(kap[0] - kappa).max() < 1e-9 * kappa
    assert np.abs(kap[1:]).max() < 1e-12 and np.abs(sig).max() < 1e-12
    av, aw = o.rhs(x, np.zeros_like(x), Q, np.zeros((3, n)))
    J = 1000 * (L / n) * I
    assert np.abs(aw).max() * J / M < 1e-8
    # nodal force residual: strain round-off (~1e-15) times the shear stiffness, in newtons
    assert np.abs(av).max() * (1000 * A * L / n) < 1e-10
    # the opposite couple is not an equilibrium of this arc
    couple[0, -1] = -M
    av, aw = Oracle(p.replace(elem_couple=couple)).rhs(x, np.zeros_like(x), Q, np.zeros((3, n)))
    assert np.abs(aw[0, -1]) * J / M > 1.0


def _settled_tip(n, L, r, F):
    E = 1e6
    A, I, EA, EI, GAs = _consts(r)
    w1 = 3.516 * np.sqrt(EI / (1000 * A * L ** 4))
    nu = 2 * 1000 * A * w1          # about critical damping of the first mode
    dt = min(1e-4, 0.1 * (L / n) / np.sqrt(E / 1000))
    steps = int(14 / w1 / dt)
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=F, nu=nu, dt=dt)
    x, v, Q, w = Oracle(p).step(*p.state(), dt=dt, n_steps=steps)
    return x[1, -1], np.abs(v).max()


@pytest.mark.parametrize("L,r", [(0.1, 0.02), (0.2, 0.01)])
def test_timoshenko_cantilever(L, r):
    """Small transverse tip load (deflection/L ~ 1e-3): the settled tip deflection converges
    at first order in 1/n to F L^3/(3EI) + F L/(alpha_c G A); Richardson extrapolation of
    n = 25, 50 lands within 0.3% (the shear term is 3.3% of the total for the stubby rod)."""
    A, I, EA, EI, GAs = _consts(r)
    F = 1e-2 * (r / 0.02) ** 4
    ref = F * L ** 3 / (3 * EI) + F * L / GAs
    d25, v25 = _settled_tip(25, L, r, F)
    d50, v50 = _settled_tip(50, L, r, F)
    e25, e50 = d25 / ref - 1, d50 / ref - 1
    assert -0.08 < e25 < -0.03 and -0.04 < e50 < -0.015
    assert 1.7 < e25 / e50 < 2.3                       # first-order convergence
    assert abs((2 * d50 - d25) / ref - 1) < 3e-3      # extrapolated limit


def _elastica_tip(L, EI, F):
    """Tip of the inextensible elastica of a cantilever under a transverse dead tip load F:
    EI theta'' + F cos(theta) = 0, theta(0) = 0, theta'(L) = 0 (theta: tangent angle from the
    clamped axis), x' = sin(theta), z' = cos(theta); boundary-value solve in scipy."""
    from scipy.integrate import solve_bvp

    def f(s, y):
        return np.vstack([y[1], -(F / EI) * np.cos(y[0]), np.sin(y[0]), np.cos(y[0])])

    def bc(ya, yb):
        return np.array([ya[0], yb[1], ya[2], ya[3]])

    s = np.linspace(0.0, L, 401)
    y0 = np.zeros((4, s.size))
    y0[3] = s
    sol = solve_bvp(f, bc, s, y0, tol=1e-10, max_nodes=100000)
    assert sol.status == 0
    return sol.y[2, -1], sol.y[3, -1]


def test_nonlinear_elastica_cantilever():
    """The cantilever workload's load (1 m, r = 1 cm, E = 1 MPa, F = 1e-2 N: F L^2/EI = 1.27) is
    far outside linear theory (F L^3/(3EI) = 0.424 m): settled, the tip deflection converges at
    first order in 1/n to the nonlinear elastica's 0.3651 m (14 % below the linear value), and
    Richardson extrapolation of n = 25, 50 lands within 1e-3 of it (extensibility and shear
    contribute ~1e-4 here)."""
    L, r, F = 1.0, 0.01, 1e-2
    A, I, EA, EI, GAs = _consts(r)
    y_ref, z_ref = _elastica_tip(L, EI, F)
    assert abs(y_ref - 0.3651) < 1e-4 and y_ref < 0.9 * F * L ** 3 / (3 * EI)
    d25, v25 = _settled_tip(25, L, r, F)
    d50, v50 = _settled_tip(50, L, r, F)
    assert v25 < 1e-5 and v50 < 1e-5                  # settled
    e25, e50 = d25 / y_ref - 1, d50 / y_ref - 1
    assert -0.07 < e25 < -0.03 and -0.035 < e50 < -0.015
    assert 1.8 < e25 / e50 < 2.2                       # first-order convergence
    assert abs((2 * d50 - d25) / y_ref - 1) < 1e-3     # extrapolated limit
