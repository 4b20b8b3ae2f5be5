"""GPU broad phase: the contact pair set of the cell-grid search equals the oracle's exhaustive
O(N^2) pair set exactly (Results, "Fibrous granular materials", Fig. 2e: the hash grid replaces
an exhaustive search and must find the same pairs).

A pair is two segments of different rods whose closest-point distance is below r_a + r_b.  Both
sides take that decision in FP64; the inputs are random, so no pair sits within rounding of the
threshold.  Cases: the tiny random placements the oracle's own cell list is pinned on (at most
200 segments, several seeds), mixed radii with single-element rods, a 200-rod packing of the
benchmark's recipe (1 mm elements, 5 mm radius) squeezed into a small box, and a packing placed
without overlap after 1000 GPU steps (collisions developed in flight, rods partly outside the
first bounding box).
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


def _gpu(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    return s


def _as_set(pairs):
    return {(int(a), int(b)) for a, b in pairs}


def _check_equal(p, x=None, v=None, s=None):
    own = s is None
    if s is None:
        s = _gpu(p)
    got, n_cand = s.contact_pairs()
    xs = p.x if x is None else x
    ref = Oracle(p, broad_phase=0).contact_pairs(xs)
    if own:
        s.close()
    assert len(ref) > 0, "the case has no contact"
    assert np.all(got[:, 0] < got[:, 1])
    assert len(_as_set(got)) == len(got), "a pair was reported twice"
    assert _as_set(got) == _as_set(ref), (len(got), len(ref))
    assert n_cand >= len(got)
    return len(ref), n_cand


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15])
def test_pair_set_equals_exhaustive_on_tiny_inputs(seed):
    # 12 rods of 1..16 elements (at most 192 segments) in a 4 cm box
    p = rodgen.random_packing(n_rods=12, nmin=1, nmax=16, box=0.04, rest_len=2e-3, radius=0.004, seed=seed,
                              allow_overlap=True, speed=0.3)
    _check_equal(p)


def test_pair_set_with_mixed_radii_and_single_element_rods():
    p = rodgen.random_packing(n_rods=60, nmin=1, nmax=3, box=0.05, rest_len=2e-3, radius=0.004, seed=21,
                              allow_overlap=True, speed=0.3)
    rng = np.random.default_rng(21)
    p = p.replace(radius=rng.uniform(0.001, 0.007, p.n_rods))
    _check_equal(p)


def test_pair_set_equals_exhaustive_on_a_200_rod_packing():
    p = rodgen.random_packing(n_rods=200, nmin=16, nmax=64, box=0.12, seed=1234, allow_overlap=True, speed=0.5)
    n, n_cand = _check_equal(p)
    assert n > 200


def test_pair_set_after_steps_on_the_gpu():
    # placed without overlap, rigid speeds up to 2 m/s, a soft dashpot: collisions develop over
    # 1000 steps with the skin list, then the grid of the moved state is searched
    p = rodgen.random_packing(n_rods=200, nmin=16, nmax=64, box=0.15, seed=99, speed=2.0).replace(contact_c=1.0)
    s = _gpu(p)
    s.contact_skin(5e-4)
    s.step(1000, 5e-6)
    x, v, Q, w = s.get_state()
    q = p.replace(x=x, v=v, Q=Q, w=w)
    _check_equal(q, s=s)
    s.close()
