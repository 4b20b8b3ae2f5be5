"""Parity at the benchmark's full size: the 10^4-rod packing (1,366,295 elements, element counts
U{16..256}) in the launch configuration bench.py times (0.5 mm skin list, the autotuner's launch
shape), element by element against the oracle.

The benchmark's own state has no contact at its start (rods placed without overlap), so the
contact checks also use the same ensemble placed with overlaps (every rod crossing several
others) and perturbed (element turns of ~0.05 rad, angular velocities, small position and
velocity noise), so that every right-hand-side term is physical; stepped, that placement uses a
softer spring (k = 10 N/m, c = 0.01 N s/m: with the benchmark's k = 1e4 its deepest overlaps
push nodes at ~3e7 m/s^2 and stretch elements past the contact grid's limit within two steps,
which the library reports as ROD_ERR_OVERFLOW).  Tolerances: 1e-12 relative
per right-hand-side array, 1e-9 of the longest rod on positions and 1e-10 relative on
velocities after the steps.  In the benchmark's own state the rods are straight and
unstressed: their couples come only from the rounding of positions near 1 m (strains of
~1e-13), so angular velocities there are compared against a floor of the velocity scale over
the element length instead of their own (noise) magnitude."""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

DT = 5e-6
SKIN = 5e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def overlapping():
    return rodgen.perturbed(rodgen.random_packing(seed=1234, allow_overlap=True), seed=5, pos=1e-3, vel=0.1,
                            rot=0.05, omega=5.0)


@pytest.fixture(scope="module")
def bench_packing():
    return rodgen.random_packing_cached(seed=1234)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _bench_system(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.contact_skin(SKIN)
    s.set_state(*p.state())
    s.autotune(DT, trial_steps=2)
    return s


def test_full_size_rhs_with_contact(overlapping):
    from paper_2605_13766_gb300 import RodSystem
    p = overlapping
    assert p.n_elems == 1366295
    o = Oracle(p)
    fc = o.contact_forces(p.x, p.v)
    assert (np.abs(fc).sum(0) > 0).sum() > 100000        # contact everywhere
    av_ref, aw_ref = o.rhs(*p.state(), t=0.0)
    s = RodSystem(p)
    s.set_state(*p.state())
    av, aw = (a.cpu().numpy() for a in s.rhs(0.0))
    assert _rel(av, av_ref) <= 1e-12
    assert _rel(aw, aw_ref) <= 1e-12
    s.close()


@pytest.mark.parametrize("which", ["bench_state", "overlapping"])
def test_full_size_steps_in_the_bench_configuration(which, overlapping, bench_packing):
    p = bench_packing if which == "bench_state" else overlapping.replace(contact_k=10.0, contact_c=0.01)
    n = 3
    ref = Oracle(p).step(*p.state(), dt=DT, n_steps=n)
    s = _bench_system(p)
    s.step(n, DT)
    got = s.get_state()
    L = float(p.n_elem.max() * p.rest_len.max())
    assert np.abs(got[0] - ref[0]).max() / L <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-10
    w_scale = max(np.abs(ref[3]).max(), np.abs(ref[1]).max() / float(p.rest_len.min()))
    assert np.abs(got[3] - ref[3]).max() <= 1e-10 * w_scale
    assert np.abs(got[2] - ref[2]).max() <= 1e-12
    s.close()
