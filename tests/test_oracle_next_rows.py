"""Oracle pins for the rows after the step: the magnetic couple of magnetized filaments
(Methods, Eq. 2), travelling-wave muscle couples, rod-wall contact with friction and rod-rod
friction.  Each is pinned by a closed form the mechanics fixes:

* a rigid-enough rod magnetized along its axis in a uniform field swings like a compass
  needle, period 2 pi sqrt(I / (M B)) (I about the centre, M = m L its moment);
* internal muscle couples tau_k at the Voronoi points bend a free rod to B kappa_k = tau_k at
  equilibrium and exert no net force;
* a one-element rod resting on a wall sinks by (m/2) g / k per node; sliding on it with
  friction mu decelerates at mu g; a wall sliding under a resting rod drags it at mu g; a wall
  moving along its normal changes the penetration by u t;
* two crossing segments in sliding contact: friction mu f_n against the sliding direction,
  split onto the nodes like the normal force, viscous below the slip velocity.
"""
import numpy as np

import rodgen
from rodgen import _straight_rods
from oracle.oracle import Oracle


def _rod(n, L, r, E=1e6, base=(0.0, 0.0, 0.0), d3=(0.0, 0.0, 1.0), ref=(1.0, 0.0, 0.0), **kw):
    n_elem = np.array([n], dtype=np.int32)
    rest = np.full(n, L / n)
    x, Q = _straight_rods(n_elem, rest, np.array([base], float), np.array([d3], float), np.array([ref], float))
    return rodgen.RodProblem(
        name="rod", n_elem=n_elem, rest_len=rest, radius=np.full(1, r), youngs=np.full(1, E),
        shear_mod=np.full(1, E / 1.5), density=np.full(1, 1000.0), x=x, v=np.zeros_like(x), Q=Q,
        w=np.zeros((3, n)), **kw)


# ---------------------------------------------------------------- magnetic couple (Eq. 2)

def _compass(th0, m0=1.0, B=0.01, n=20, L=0.1, r=0.002, E=1e8):
    d3 = np.array([np.cos(th0), np.sin(th0), 0.0])
    return _rod(n, L, r, E=E, base=tuple(-0.5 * L * d3), d3=tuple(d3), ref=(0.0, 0.0, 1.0),
                magnetization=np.tile(np.array([[0.0], [0.0], [m0]]), (1, n)),
                field_b0=np.array([B, 0.0, 0.0]))


def test_magnetized_rod_swings_like_a_compass_needle():
    th0, m0, B, n, L, r = 0.05, 1.0, 0.01, 20, 0.1, 0.002
    p = _compass(th0, m0, B, n, L, r)
    A, I1 = np.pi * r * r, np.pi * r ** 4 / 4
    I_tot = 1000 * A * L ** 3 / 12 + 1000 * I1 * L
    T = 2 * np.pi * np.sqrt(I_tot / (m0 * L * B))
    dt, chunk = 2e-6, 250
    o = Oracle(p)
    st = p.state()
    t, ts, ang = 0.0, [0.0], [th0]
    while t < 0.8 * T:
        st = o.step(*st, dt=dt, n_steps=chunk, t=t)
        t += chunk * dt
        x = st[0]
        ts.append(t)
        ang.append(np.arctan2(x[1, -1] - x[1, 0], x[0, -1] - x[0, 0]))
    ts, ang = np.array(ts), np.array(ang)
    assert ang[1] < th0                      # turns toward the field (a flipped couple would turn away)
    # zero crossings at T/4 and 3T/4
    zc = [ts[i] - ang[i] * (ts[i + 1] - ts[i]) / (ang[i + 1] - ang[i])
          for i in range(len(ang) - 1) if ang[i] > 0 >= ang[i + 1] or ang[i] < 0 <= ang[i + 1]]
    assert len(zc) >= 2
    T_meas = 2 * (zc[1] - zc[0])
    assert abs(T_meas / T - 1) < 0.01, (T_meas, T)
    assert abs(zc[0] / (T / 4) - 1) < 0.01
    assert abs(np.abs(ang).max() / th0 - 1) < 0.02   # the swing keeps its amplitude


def test_field_along_the_magnetization_exerts_no_couple():
    p = _compass(0.0)                          # rod and field both along x, m along d3
    _, aw = Oracle(p).rhs(*p.state())
    assert np.abs(aw).max() == 0.0
    q = _compass(0.3)
    _, aw = Oracle(q).rhs(*q.state())
    # |couple| = rl m B sin(th) about d1 (= z), towards the field: negative about +z
    r, L, n = 0.002, 0.1, 20
    rl, I1 = L / n, np.pi * r ** 4 / 4
    expect = -rl * 1.0 * 0.01 * np.sin(0.3) / (1000 * I1 * rl)
    # (rounding-level internal couples of the straight rod at 0.3 rad remain: 1e-9)
    assert np.allclose(aw[0], expect, rtol=1e-9) and np.abs(aw[1:]).max() < 1e-9 * abs(expect)


# ---------------------------------------------------------------- travelling-wave muscle couples

def test_muscle_couples_bend_a_free_rod_to_tau_over_B():
    n, L, r, E = 40, 0.2, 0.005, 1e6
    A, I1 = np.pi * r * r, np.pi * r ** 4 / 4
    Am, lam, phi = 1e-5, 0.2, 0.7
    w1 = 22.4 * np.sqrt(E * I1 / (1000 * A * L ** 4))     # first free-free bending mode
    nu = 2 * 1000 * A * w1
    p = _rod(n, L, r, E=E, d3=(1.0, 0.0, 0.0), ref=(0.0, 0.0, 1.0), nu_damp=nu,
             muscle_amp=np.full(1, Am), muscle_period=np.full(1, 1e9), muscle_wavelength=np.full(1, lam),
             muscle_phase=np.full(1, phi))
    dt = 0.1 * (L / n) / np.sqrt(E / 1000)
    o = Oracle(p)
    x, v, Q, w = o.step(*p.state(), dt=dt, n_steps=int(16 / w1 / dt))
    assert np.abs(v).max() < 1e-6
    _, kap, _, _ = o.strains(x, Q)
    s = np.arange(1, n) * (L / n)
    tau = Am * np.sin(-2 * np.pi * s / lam + phi)
    B1 = E * I1
    err = np.abs(kap[0] - tau / B1).max() / np.abs(tau / B1).max()
    assert err < 0.01, err
    # no net force: the centre of mass has not moved
    m = np.full(n + 1, 1.0)
    m[[0, -1]] = 0.5
    com0 = (p.x * m).sum(axis=1) / m.sum()
    com = (x * m).sum(axis=1) / m.sum()
    assert np.abs(com - com0).max() < 1e-12


def test_muscle_couples_are_internal():
    """Planar muscles (d1 = lab z) on a free rod at rest: linear momentum stays zero and the
    angular momentum about z stays at rounding level while the rod moves."""
    n, L, r = 30, 0.2, 0.005
    p = _rod(n, L, r, d3=(1.0, 0.0, 0.0), ref=(0.0, 0.0, 1.0), muscle_amp=np.full(1, 1e-4),
             muscle_period=np.full(1, 0.05), muscle_wavelength=np.full(1, 0.1), muscle_phase=np.zeros(1))
    o = Oracle(p)
    x, v, Q, w = o.step(*p.state(), dt=1e-5, n_steps=2000)
    A = np.pi * r * r
    m = np.full(n + 1, 1000 * A * L / n)
    m[[0, -1]] *= 0.5
    P = (v * m).sum(axis=1)
    assert np.abs(v).max() > 1e-4                       # it moves
    assert np.abs(P).max() < 1e-15 * m.sum() * 1e3
    I1 = np.pi * r ** 4 / 4
    # orbital part plus the elements' spin about d1 (= lab z): rho I1 rl w_1
    Lz = (np.cross(x.T, (v * m).T)[:, 2]).sum() + (1000 * I1 * (L / n) * w[0]).sum()
    scale = m.sum() * np.abs(v).max() * L
    assert abs(Lz) < 1e-6 * scale


# ---------------------------------------------------------------- walls

def _segment_on_ground(r=0.005, ell=0.01, k=100.0, c=None, mu=0.0, vslip=1e-6, u=(0.0, 0.0, 0.0), z0=None,
                       vx=0.0, g=9.81):
    m_node = 0.5 * 1000 * np.pi * r * r * ell
    c = 2 * np.sqrt(k * m_node) if c is None else c
    z = r if z0 is None else z0
    p = _rod(1, ell, r, d3=(1.0, 0.0, 0.0), ref=(0.0, 0.0, 1.0), base=(0.0, 0.0, z),
             gravity=np.array([0.0, 0.0, -g]), wall_point=np.zeros((1, 3)), wall_normal=np.array([[0.0, 0.0, 1.0]]),
             wall_velocity=np.array([u]), wall_k=k, wall_c=c, wall_mu=mu, wall_vslip=vslip)
    p.v[0, :] = vx
    return p, m_node


def test_segment_resting_on_a_wall_sinks_by_mg_over_k():
    r, k, g = 0.005, 100.0, 9.81
    p, m_node = _segment_on_ground(r=r, k=k)
    x, v, Q, w = Oracle(p).step(*p.state(), dt=1e-5, n_steps=4000)
    delta = m_node * g / k
    assert np.abs(v).max() < 1e-8
    assert np.allclose(x[2], r - delta, rtol=0, atol=1e-6 * delta)
    # a wall pushing the wrong way (or a missing radius) would let it fall through or float


def test_sliding_on_a_wall_decelerates_at_mu_g():
    r, k, g, mu, v0 = 0.005, 100.0, 9.81, 0.3, 0.1
    p, m_node = _segment_on_ground(r=r, k=k, mu=mu, vx=v0)
    p.x[2, :] = r - m_node * g / k                # start at the resting penetration
    t = 0.01
    x, v, Q, w = Oracle(p).step(*p.state(), dt=1e-5, n_steps=int(round(t / 1e-5)))
    assert np.allclose(v[0], v0 - mu * g * t, rtol=1e-6)
    assert np.abs(v[2]).max() < 1e-9


def test_a_wall_sliding_under_a_resting_rod_drags_it_at_mu_g():
    r, k, g, mu, u = 0.005, 100.0, 9.81, 0.2, 0.5
    p, m_node = _segment_on_ground(r=r, k=k, mu=mu, u=(u, 0.0, 0.0))
    p.x[2, :] = r - m_node * g / k
    t = 0.01
    x, v, Q, w = Oracle(p).step(*p.state(), dt=1e-5, n_steps=int(round(t / 1e-5)))
    assert np.allclose(v[0], mu * g * t, rtol=1e-6)          # still slower than the wall


def test_a_wall_moving_along_its_normal_changes_the_penetration():
    r, k = 0.005, 100.0
    u = 0.01
    p, m_node = _segment_on_ground(r=r, k=k, c=0.0, u=(0.0, 0.0, u), z0=r - 1e-4, g=0.0)
    o = Oracle(p)
    a0, _ = o.rhs(*p.state(), t=0.0)
    a1, _ = o.rhs(*p.state(), t=2e-3)
    # the penetration grows by u t, the force by k u t on each node
    assert np.allclose((a1[2] - a0[2]) * m_node, k * u * 2e-3, rtol=1e-9)
    assert np.allclose(a0[2] * m_node, k * 1e-4, rtol=1e-9)


# ---------------------------------------------------------------- rod-rod friction

def _crossing_sliding(d, r=0.005, ell=0.004, vb=(0.0, 0.0, 0.0), mu=0.0, vslip=1e-6, shift=0.0):
    n_elem = np.array([1, 1], dtype=np.int32)
    x = np.array([[-ell / 2, ell / 2, shift, shift],
                  [0.0, 0.0, -ell / 2, ell / 2],
                  [0.0, 0.0, d, d]])
    v = np.zeros((3, 4))
    v[:, 2:4] = np.array(vb)[:, None]
    Q = np.array([[0.0, 1.0], [1.0, 0.0], [0.0, 0.0],
                  [0.0, 0.0], [0.0, 0.0], [-1.0, -1.0],
                  [1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    return rodgen.RodProblem(
        name="crossing", n_elem=n_elem, rest_len=np.full(2, ell), radius=np.full(2, r),
        youngs=np.full(2, 1e6), shear_mod=np.full(2, 1e6 / 1.5), density=np.full(2, 1000.0),
        x=x, v=v, Q=Q, w=np.zeros((3, 2)), contact=True, contact_k=1e4, contact_c=10.0,
        contact_mu=mu, contact_vslip=vslip)


def test_sliding_crossing_feels_coulomb_friction():
    r, d, k, mu, wv = 0.005, 0.006, 1e4, 0.4, 0.3
    F = k * (2 * r - d)
    # B (above) slides along +x over A: A is dragged along +x, B held back
    q = _crossing_sliding(d, r=r, vb=(wv, 0.0, 0.0), mu=mu, shift=0.001)
    f = Oracle(q).contact_forces(q.x, q.v)
    fa, fb = f[:, 0:2].sum(axis=1), f[:, 2:4].sum(axis=1)
    assert np.allclose(fa, [mu * F, 0.0, -F], rtol=1e-12, atol=1e-12 * F)
    assert np.allclose(fb, -fa, rtol=1e-12, atol=1e-12 * F)
    # split like the normal force: A's nodes 1/4 : 3/4 (contact at s = 3/4)
    assert np.allclose(f[0, 0:2], [0.25 * mu * F, 0.75 * mu * F], rtol=1e-12)
    # below the slip velocity the friction is viscous: mu F v / v_slip
    q = _crossing_sliding(d, r=r, vb=(2e-7, 0.0, 0.0), mu=mu, vslip=1e-6)
    f = Oracle(q).contact_forces(q.x, q.v)
    assert np.isclose(f[0, 0:2].sum(), mu * F * 0.2, rtol=1e-9)
    # sliding along the normal only (approach): no tangential force
    q = _crossing_sliding(d, r=r, vb=(0.0, 0.0, -0.1), mu=mu)
    f = Oracle(q).contact_forces(q.x, q.v)
    assert np.abs(f[0:2]).max() < 1e-12 * F
    # mu = 0: the frictionless force
    q = _crossing_sliding(d, r=r, vb=(wv, 0.0, 0.0), mu=0.0)
    f = Oracle(q).contact_forces(q.x, q.v)
    assert np.abs(f[0:2]).max() == 0.0
