"""GPU parity of rod-rod contact (cell-list broad phase + FP64 narrow phase) against the oracle.

The oracle's exhaustive O(N^2) search is the reference for the pair set; its forces are
compared element by element (relative 1e-12), then the right-hand side with contact and short
trajectories through collisions.
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _dense(n_rods=80, box=0.08, seed=1, nmin=3, nmax=30, speed=0.3):
    return rodgen.random_packing(n_rods=n_rods, nmin=nmin, nmax=nmax, box=box, rest_len=2e-3, radius=0.004,
                                 seed=seed, allow_overlap=True, speed=speed)


def _gpu(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    return s


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_contact_forces_match_exhaustive_oracle(seed):
    p = _dense(seed=seed)
    o = Oracle(p, broad_phase=0)
    ref = o.contact_forces(p.x, p.v)
    got = _gpu(p).contact_forces().cpu().numpy()
    assert np.abs(ref).max() > 1.0            # there is contact
    assert _rel(got, ref) <= 1e-12, _rel(got, ref)
    assert np.abs(got.sum(1)).max() <= 1e-11 * np.abs(ref).max()


def test_contact_forces_with_mixed_radii_and_single_element_rods():
    p = _dense(n_rods=60, nmin=1, nmax=6, seed=7)
    rng = np.random.default_rng(7)
    p = p.replace(radius=rng.uniform(0.002, 0.006, p.n_rods))
    ref = Oracle(p, broad_phase=0).contact_forces(p.x, p.v)
    got = _gpu(p).contact_forces().cpu().numpy()
    assert np.abs(ref).max() > 1.0
    assert _rel(got, ref) <= 1e-12


def test_rhs_with_contact_matches_oracle():
    p = _dense(seed=4).replace(gravity=np.array([0.0, 0.0, -9.81]))
    p = rodgen.perturbed(p, seed=5, pos=0.01, rot=0.02)
    o = Oracle(p)
    av_ref, aw_ref = o.rhs(*p.state(), t=0.0)
    av, aw = (a.cpu().numpy() for a in _gpu(p).rhs(0.0))
    assert _rel(av, av_ref) <= 1e-12 and _rel(aw, aw_ref) <= 1e-12


def _touching(n_rods, box, seed, nmin=8, nmax=40, speed=1.0):
    """Rods placed without deep overlap (at most 1 mm) so that contact acts from the first step."""
    return rodgen.random_packing(n_rods=n_rods, nmin=nmin, nmax=nmax, box=box, rest_len=2e-3, radius=0.004,
                                 seed=seed, speed=speed, dt=2e-6, margin=-1e-3)


def test_trajectory_through_collisions():
    """400 steps of rods pressed into each other (overlaps up to 1 mm) and moving."""
    p = _touching(40, 0.08, 6)
    o = Oracle(p)
    assert np.abs(o.contact_forces(p.x, p.v)).max() > 0.5      # contact acts from the start
    ref = o.step(*p.state(), dt=2e-6, n_steps=400)
    s = _gpu(p)
    s.step(400, 2e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() / 0.08 <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7


def test_trajectory_with_contact_200_rods_1000_steps():
    p = _touching(200, 0.2, 12, nmin=16, nmax=64)
    o = Oracle(p)
    assert np.abs(o.contact_forces(p.x, p.v)).max() > 0.5
    ref = o.step(*p.state(), dt=2e-6, n_steps=1000)
    s = _gpu(p)
    s.step(1000, 2e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() / 0.128 <= 1e-9


def test_graph_replay_equals_eager_launches():
    """100 contact steps: replayed CUDA graphs (32 steps each) and eager launches agree, and both
    match the oracle."""
    p = _touching(60, 0.1, 14)
    ref = Oracle(p).step(*p.state(), dt=2e-6, n_steps=100)
    a = _gpu(p)
    a.step(100, 2e-6)
    b = _gpu(p)
    b.use_graphs(False)
    b.step(100, 2e-6)
    ga, gb = a.get_state(), b.get_state()
    assert np.abs(ga[0] - gb[0]).max() <= 1e-15
    assert np.abs(ga[0] - ref[0]).max() / 0.1 <= 1e-9
    assert a.launch_count > 0


def test_element_longer_than_the_grid_allows_is_reported():
    from paper_2605_13766_gb300 import RodError
    p = _dense(n_rods=10, seed=9, nmin=4, nmax=8)
    x, v, Q, w = p.state()
    # pull every rod apart along its axis: elements grow far beyond the twice their length the
    # grid covers
    off = p.node_offsets()
    for r in range(p.n_rods):
        a, b = off[r], off[r + 1]
        c = x[:, a:b].mean(1, keepdims=True)
        v[:, a:b] = 10000.0 * (x[:, a:b] - c)
    q = p.replace(v=v, contact_k=0.0, contact_c=0.0)
    s = _gpu(q)
    with pytest.raises(RodError) as ei:
        s.step(400, 1e-6)
    assert ei.value.status == -5
