"""Oracle pins for rod-rod contact (broad phase and narrow phase).

* segment-segment closest points: the returned pair attains the minimum distance over
  [0,1]^2, checked against a dense (s, u) grid refined by a bounded quasi-Newton search;
* the uniform cell list proposes exactly the pairs that the exhaustive O(N^2) search finds in
  contact (results section, exhaustive search vs hash grid), including stretched segments that
  enlarge the cell size;
* Newton's third law: contact forces sum to zero; both broad phases give the same forces;
* closed form: two perpendicular crossing segments at centre distance d < 2r push each other
  apart with k (2r - d), split evenly; an approach speed adds c u; a fast separation clamps to 0.
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle, segment_closest

optimize = pytest.importorskip("scipy.optimize")


def _dist(p0, p1, q0, q1, s, u):
    return np.linalg.norm(p0 + s * (p1 - p0) - (q0 + u * (q1 - q0)))


def _reference_min(p0, p1, q0, q1):
    g = np.linspace(0.0, 1.0, 201)
    S, U = np.meshgrid(g, g, indexing="ij")
    P = p0[None, None, :] + S[..., None] * (p1 - p0)
    R = q0[None, None, :] + U[..., None] * (q1 - q0)
    D = np.linalg.norm(P - R, axis=-1)
    i, j = np.unravel_index(np.argmin(D), D.shape)
    f = lambda z: _dist(p0, p1, q0, q1, z[0], z[1]) ** 2
    res = optimize.minimize(f, [g[i], g[j]], method="L-BFGS-B", bounds=[(0, 1), (0, 1)],
                            options={"ftol": 1e-30, "gtol": 1e-16, "maxiter": 500})
    return min(np.sqrt(res.fun), D.min())


def _cases(rng):
    cases = []
    for _ in range(150):
        cases.append(tuple(rng.uniform(-1, 1, (4, 3))))
    for _ in range(30):  # short segments (the workload's aspect), nearby
        c = rng.uniform(-0.01, 0.01, 3)
        a, b = rng.normal(size=3), rng.normal(size=3)
        a *= 1e-3 / np.linalg.norm(a)
        b *= 1e-3 / np.linalg.norm(b)
        cases.append((np.zeros(3), a, c, c + b))
    d = np.array([1.0, 0.2, -0.3])
    cases.append((np.zeros(3), d, np.array([0.1, 0.5, 0.0]), np.array([0.1, 0.5, 0.0]) + d))       # parallel
    cases.append((np.zeros(3), d, np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.5, 0.0]) + d * (1 + 1e-12)))
    cases.append((np.zeros(3), d, 2 * d, 3 * d))                                                   # collinear gap
    cases.append((np.zeros(3), np.array([1.0, 0, 0]), np.array([0.5, -1.0, 0.3]), np.array([0.5, 1.0, 0.3])))
    cases.append((np.zeros(3), np.array([1.0, 0, 0]), np.array([1.0, 0, 0]), np.array([2.0, 1.0, 0.0])))  # touching ends
    return cases


def test_segment_closest_attains_minimum():
    rng = np.random.default_rng(8)
    for p0, p1, q0, q1 in _cases(rng):
        s, u = segment_closest(p0, p1, q0, q1)
        assert 0.0 <= s <= 1.0 and 0.0 <= u <= 1.0
        d_alg = _dist(p0, p1, q0, q1, s, u)
        d_ref = _reference_min(p0, p1, q0, q1)
        scale = max(np.linalg.norm(p1 - p0), np.linalg.norm(q1 - q0))
        assert d_alg <= d_ref + 1e-9 * scale, (d_alg, d_ref)


def test_parallel_tie_break():
    """Parallel segments start from s = 0; u = -0.25 is clamped to 0 and s re-solved to 0.25,
    which is one of the (non-unique) minimisers at distance 1."""
    d = np.array([1.0, 0.0, 0.0])
    s, u = segment_closest(np.zeros(3), d, np.array([0.25, 1.0, 0.0]), np.array([1.25, 1.0, 0.0]))
    assert (s, u) == (0.25, 0.0)
    s, u = segment_closest(np.zeros(3), d, np.array([-0.5, 1.0, 0.0]), np.array([0.5, 1.0, 0.0]))
    assert (s, u) == (0.0, 0.5)


def _packing(n_rods, box, seed, stretch=1.0):
    p = rodgen.random_packing(n_rods=n_rods, nmin=3, nmax=12, box=box, rest_len=2e-3, radius=0.004,
                              seed=seed, allow_overlap=True, speed=0.3)
    if stretch != 1.0:
        x = p.x.copy()
        off = p.node_offsets()
        for r in range(p.n_rods):
            a, b = off[r], off[r + 1]
            x[:, a:b] = x[:, a:a + 1] + stretch * (x[:, a:b] - x[:, a:a + 1])
        p = p.replace(x=x)
    return p


@pytest.mark.parametrize("seed,stretch", [(1, 1.0), (2, 1.0), (3, 2.5)])
def test_cell_list_pairs_equal_exhaustive(seed, stretch):
    p = _packing(60, 0.06, seed, stretch)
    o = Oracle(p, broad_phase=0)
    brute = o.contact_pairs(p.x)
    o.set_broad_phase(1)
    cells = o.contact_pairs(p.x)
    assert len(brute) > 20
    assert set(map(tuple, brute)) == set(map(tuple, cells))
    assert len(cells) == len(set(map(tuple, cells)))


def test_contact_forces_balance_and_match_between_broad_phases():
    p = _packing(60, 0.06, 5)
    o = Oracle(p, broad_phase=0)
    fb = o.contact_forces(p.x, p.v)
    o.set_broad_phase(1)
    fc = o.contact_forces(p.x, p.v)
    scale = np.abs(fb).max()
    assert scale > 1.0
    assert np.abs(fb.sum(1)).max() < 1e-12 * scale * p.n_nodes
    assert np.abs(fb - fc).max() < 1e-12 * scale


def _crossing(d, r=0.005, ell=0.004, va=0.0, vb=0.0, shift=0.0):
    """Rod A along x at z = 0, rod B along y at z = d crossing A at x = shift; one element each."""
    n_elem = np.array([1, 1], dtype=np.int32)
    x = np.array([[-ell / 2, ell / 2, shift, shift],
                  [0.0, 0.0, -ell / 2, ell / 2],
                  [0.0, 0.0, d, d]])
    v = np.zeros((3, 4))
    v[2, 0:2] = va
    v[2, 2:4] = vb
    Q = np.array([[0.0, 1.0], [1.0, 0.0], [0.0, 0.0],      # d1
                  [0.0, 0.0], [0.0, 0.0], [-1.0, -1.0],   # d2 = d3 x d1
                  [1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])    # d3 (A: x, B: y)
    return rodgen.RodProblem(
        name="crossing", n_elem=n_elem, rest_len=np.full(2, ell), radius=np.full(2, r),
        youngs=np.full(2, 1e6), shear_mod=np.full(2, 1e6 / 1.5), density=np.full(2, 1000.0),
        x=x, v=v, Q=Q, w=np.zeros((3, 2)), contact=True, contact_k=1e4, contact_c=10.0)


def test_crossing_segments_closed_form():
    r, d, k, c = 0.005, 0.006, 1e4, 10.0
    p = _crossing(d, r=r)
    o = Oracle(p)
    f = o.contact_forces(p.x, p.v)
    F = k * (2 * r - d)
    expect = np.zeros((3, 4))
    expect[2, 0:2] = -F / 2       # A is below B: pushed toward -z
    expect[2, 2:4] = +F / 2
    assert np.abs(f - expect).max() < 1e-12 * F
    # approaching at speed u adds c u
    u = 0.2
    q = _crossing(d, r=r, va=u)
    f = Oracle(q).contact_forces(q.x, q.v)
    assert abs(f[2, 0] - (-(F + c * u) / 2)) < 1e-12 * F
    # separating faster than k delta / c: no (attractive) force
    q = _crossing(d, r=r, va=-5.0)      # c u = 50 N > k delta = 40 N
    f = Oracle(q).contact_forces(q.x, q.v)
    assert np.abs(f).max() == 0.0
    # out of reach: no force
    q = _crossing(2 * r + 1e-6, r=r)
    assert np.abs(Oracle(q).contact_forces(q.x, q.v)).max() == 0.0
    # crossing at s = 3/4 of A: A's nodes share the force 1/4 : 3/4
    q = _crossing(d, r=r, shift=0.001)
    f = Oracle(q).contact_forces(q.x, q.v)
    assert abs(f[2, 0] - (-0.25 * F)) < 1e-12 * F and abs(f[2, 1] - (-0.75 * F)) < 1e-12 * F
