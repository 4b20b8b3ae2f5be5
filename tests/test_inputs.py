"""The seeded synthetic inputs follow their stated recipes (CPU).

* the exact axis-segment distance used for placement agrees with brute-force sampling;
* a random packing placed without overlap keeps every pair of rods of different axes at least
  2 r + margin apart (all pairs, exact distances), and its lengths, speeds and frames follow
  the recipe (n ~ U{nmin..nmax}, rigid velocity per rod within [-speed, speed]^3, orthonormal
  frames with d3 along the rod);
* the cilia carpet: upright clamped rods on the square grid, base couple amplitude 0.5 E I / L;
* the adjoint batch: the stated distributions of rest curvature, couples and tip targets;
* the same seed gives the same arrays;
* a sub-ensemble taken out of an ensemble (the reference arm's bounded samples) is the same rods.
"""
import numpy as np
import pytest

import rodgen
from rodgen import _axis_distance


def test_axis_distance_against_sampling():
    rng = np.random.default_rng(0)
    m = 40
    c1, c2 = rng.normal(0, 0.5, (m, 3)), rng.normal(0, 0.5, (m, 3))
    a1, a2 = rng.normal(size=(m, 3)), rng.normal(size=(m, 3))
    a1 /= np.linalg.norm(a1, axis=1, keepdims=True)
    a2 /= np.linalg.norm(a2, axis=1, keepdims=True)
    a2[:5] = a1[:5]                                  # parallel pairs
    h1, h2 = rng.uniform(0.05, 1.0, m), rng.uniform(0.05, 1.0, m)
    got = _axis_distance(c1, a1, h1, c2, a2, h2)
    s = np.linspace(-1.0, 1.0, 801)
    for k in range(m):
        p = c1[k] + (s * h1[k])[:, None] * a1[k]
        q = c2[k] + (s * h2[k])[:, None] * a2[k]
        brute = np.sqrt(((p[:, None, :] - q[None, :, :]) ** 2).sum(-1)).min()
        # sampling at spacing h/400 overestimates the minimum by at most (h1 + h2) / 400
        assert got[k] <= brute + 1e-12
        assert got[k] >= brute - (h1[k] + h2[k]) / 400.0


def _axes(p):
    no = p.node_offsets()
    first, last = p.x[:, no[:-1]].T, p.x[:, no[1:] - 1].T
    c = 0.5 * (first + last)
    d = last - first
    h = 0.5 * np.linalg.norm(d, axis=1)
    return c, d / (2 * h[:, None]), h


def test_packing_without_overlap_follows_the_recipe():
    R, radius, margin, speed = 150, 0.005, 5e-4, 0.5
    p = rodgen.random_packing(n_rods=R, nmin=16, nmax=256, box=0.5, radius=radius, margin=margin, speed=speed,
                              seed=11)
    assert p.n_rods == R and p.n_elem.min() >= 16 and p.n_elem.max() <= 256
    assert np.allclose(p.rest_len, 1e-3)
    c, a, h = _axes(p)
    i, j = np.triu_indices(R, 1)
    d = _axis_distance(c[i], a[i], h[i], c[j], a[j], h[j])
    assert d.min() >= 2 * radius + margin - 1e-9, d.min()
    # rigid velocity per rod, within the stated cube
    no = p.node_offsets()
    for r in range(R):
        v = p.v[:, no[r]:no[r + 1]]
        assert np.allclose(v, v[:, :1]) and np.abs(v).max() <= speed
    # orthonormal frames, d3 along the rod
    Q = p.Q.reshape(3, 3, -1)
    G = np.einsum("aie,bie->abe", Q, Q)
    assert np.abs(G - np.eye(3)[:, :, None]).max() < 1e-12
    eo = p.elem_offsets()
    for r in range(R):
        assert np.allclose(Q[2][:, eo[r]:eo[r + 1]], a[r][:, None], atol=1e-12)


def test_packing_is_seeded():
    a = rodgen.random_packing(n_rods=40, box=0.3, seed=5)
    b = rodgen.random_packing(n_rods=40, box=0.3, seed=5)
    c = rodgen.random_packing(n_rods=40, box=0.3, seed=6)
    for name in ("n_elem", "x", "v", "Q"):
        assert np.array_equal(getattr(a, name), getattr(b, name))
    assert not np.array_equal(a.n_elem, c.n_elem)


def test_cilia_carpet_recipe():
    side, n, L, r, E = 8, 50, 0.2, 0.005, 1e6
    p = rodgen.cilia_carpet(side=side, n=n, length=L, radius=r, youngs=E, spacing=0.05)
    assert p.n_rods == side * side and np.all(p.n_elem == n)
    assert np.all(p.clamp_base == 1)
    no = p.node_offsets()
    base = p.x[:, no[:-1]]
    assert np.allclose(np.sort(np.unique(np.round(base[0], 12))), np.arange(side) * 0.05)
    assert np.allclose(base[2], 0.0)
    tips = p.x[:, no[1:] - 1]
    assert np.allclose(tips[2], L) and np.allclose(tips[:2], base[:2])      # upright
    I = np.pi * r ** 4 / 4
    assert np.allclose(p.act_amp, 0.5 * E * I / L)
    assert np.all((p.act_phase >= 0) & (p.act_phase < 2 * np.pi))
    assert np.allclose(p.shear_mod, E / 1.5)


@pytest.mark.parametrize("n", [1, 7, 100])
def test_cantilever_recipe(n):
    p = rodgen.cantilever(n=n, length=1.0, tip_force=1e-2)
    assert p.n_rods == 1 and p.n_elem[0] == n
    assert np.allclose(p.x[2], np.linspace(0.0, 1.0, n + 1)) and np.allclose(p.x[:2], 0.0)
    assert np.allclose(p.tip_force[:, 0], [0.0, 1e-2, 0.0])


def test_take_rods_matches_the_full_ensemble():
    """Without contact the rods are independent: the oracle's right-hand side of rods r0..r1-1
    taken on their own equals the matching slice of the full right-hand side, bit for bit."""
    from oracle.oracle import Oracle
    rng = np.random.default_rng(3)
    p = rodgen.perturbed(rodgen.random_packing(n_rods=12, nmin=1, nmax=40, box=0.5, seed=3, allow_overlap=True,
                                               speed=0.2), seed=3)
    p = p.replace(contact=False, tip_force=rng.normal(0, 1e-3, (3, 12)), rest_sigma=rng.normal(0, 1e-3, (3, p.n_elems)),
                  rest_kappa=rng.normal(0, 0.3, (3, p.n_voronoi)), elem_couple=rng.normal(0, 1e-6, (3, p.n_elems)),
                  clamp_base=(np.arange(12) % 3 == 0).astype(np.int8), gravity=np.array([0.0, 0.0, -9.81]))
    av, aw = Oracle(p).rhs(*p.state(), t=0.01)
    eo, no = p.elem_offsets(), p.node_offsets()
    for r0, r1 in [(0, 1), (3, 8), (11, 12), (0, 12)]:
        q = p.take_rods(r0, r1)
        bv, bw = Oracle(q).rhs(*q.state(), t=0.01)
        assert np.array_equal(bv, av[:, no[r0]:no[r1]]) and np.array_equal(bw, aw[:, eo[r0]:eo[r1]])
    with pytest.raises(ValueError):
        p.take_rods(5, 5)


def test_adjoint_batch_recipe():
    """1024 clamped upright rods x 64 elements, rest curvature ~ N(0, 0.5) 1/m, element couples
    ~ N(0, 1e-6) N m, tip targets = undeformed tips + N(0, 0.01) m (sample moments of the
    seeded draws within a few standard errors)."""
    p = rodgen.adjoint_batch()
    R, n = 1024, 64
    assert p.n_rods == R and np.all(p.n_elem == n) and np.all(p.clamp_base == 1)
    assert p.rest_kappa.shape == (3, R * (n - 1)) and p.elem_couple.shape == (3, R * n)
    k, c = p.rest_kappa.ravel(), p.elem_couple.ravel()
    assert abs(k.mean()) < 4 * 0.5 / np.sqrt(k.size) and abs(k.std() / 0.5 - 1) < 0.01
    assert abs(c.mean()) < 4 * 1e-6 / np.sqrt(c.size) and abs(c.std() / 1e-6 - 1) < 0.01
    tips = p.x[:, p.node_offsets()[1:] - 1]
    dev = (p.extra["targets"] - tips).ravel()
    assert abs(dev.std() / 0.01 - 1) < 0.05 and np.allclose(tips[2], 0.2)
