"""The step kernels compiled for a feature set against the general kernel.

The host launches the kernel of the smallest compiled feature set that covers the system: the
plain step (circular sections without rest strain or curvature, no loads but gravity and
contact), the driven-rod step (actuation couples and damping) or the general step.  The two
specialised kernels are the general kernel's arithmetic with the tests of absent features made
false at compile time, so on the same system they must agree with it bit for bit.  Element
couples that are all zero select the general kernel without changing any value (adding 0.0
changes at most the sign of a zero, which the comparison treats as equal).
"""
import numpy as np
import pytest

import rodgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _run(p, steps, dt, shape=None):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    if shape is not None:
        s.set_launch(*shape)
    s.set_state(*p.state())
    s.step(steps, dt)
    out = s.get_state()
    s.close()
    return out


def _with_zero_couples(p):
    return p.replace(elem_couple=np.zeros((3, p.n_elems)))


def _same(a, b):
    for x, y in zip(a, b):
        assert np.all(np.isfinite(x))
        assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [None, (256, 128)], ids=["default-shape", "256x128"])
def test_plain_step_with_contact_equals_the_general_kernel(shape):
    """Free rods under gravity in contact from the first step (one launch per step, skin list)."""
    p = rodgen.random_packing(n_rods=60, nmin=8, nmax=40, box=0.1, rest_len=2e-3, radius=0.004, seed=14,
                              speed=1.0, dt=2e-6, margin=-1e-3)
    _same(_run(p, 60, 2e-6, shape), _run(_with_zero_couples(p), 60, 2e-6, shape))


def test_plain_step_without_contact_equals_the_general_kernel():
    """Free rods of ragged lengths under gravity (all steps of a call in one launch)."""
    p = rodgen.random_packing(n_rods=40, nmin=1, nmax=90, box=1.0, rest_len=4e-3, radius=0.004, seed=5,
                              allow_overlap=True, speed=0.3, spin=20.0).replace(contact=False)
    _same(_run(p, 300, 5e-6), _run(_with_zero_couples(p), 300, 5e-6))


def test_driven_step_equals_the_general_kernel():
    """The cilia carpet: clamped rods with actuation couples and drag."""
    p = rodgen.cilia_carpet(side=5, n=50)
    _same(_run(p, 300, 1e-5), _run(_with_zero_couples(p), 300, 1e-5))
