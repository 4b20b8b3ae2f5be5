"""The allocation-free contact entry point (rod_contact_forces_noalloc) against the system's own
contact forces (rod_system_contact_forces) on the same states.

The entry point exists for callers that cannot allocate device memory when they need contact
forces (code running inside another framework's allocator or memory pool, loops that must stay
out of the driver's allocator); it keeps every temporary in a fixed file-scope device array.
Two calls in a row on different states check that what the array keeps from the previous
call does not leak into the next one.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import rodgen

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _system_forces(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    f = s.contact_forces().cpu().numpy()
    s.close()
    return f


def _noalloc_forces(p, f_out=None):
    import torch
    from paper_2605_13766_gb300.binding import contact_forces_noalloc
    node_off = torch.tensor(p.node_offsets().astype(np.int32), device="cuda")
    radius = torch.tensor(p.radius, device="cuda")
    x = torch.tensor(p.x, device="cuda")
    v = torch.tensor(p.v, device="cuda")
    f = torch.full((3, p.n_nodes), float("nan"), dtype=torch.float64, device="cuda") if f_out is None else f_out
    contact_forces_noalloc(node_off, radius, x, v, p.contact_k, p.contact_c, p.cell_size, f)
    return f.cpu().numpy()


def _packing(seed, n_rods=80, box=0.08):
    return rodgen.random_packing(n_rods=n_rods, nmin=3, nmax=30, box=box, rest_len=2e-3, radius=0.004, seed=seed,
                                 allow_overlap=True, speed=0.3)


def test_two_calls_in_a_row_match_the_system_entry_point():
    first = _packing(21)
    second = rodgen.perturbed(_packing(22, n_rods=120, box=0.1), seed=3, pos=0.05, vel=0.5, rot=0.0, omega=0.0)
    for p in (first, second):
        ref = _system_forces(p)
        got = _noalloc_forces(p)
        scale = np.abs(ref).max()
        assert scale > 1.0                      # there is contact to compare
        assert np.abs(got - ref).max() <= TOL * scale


def test_sizes_beyond_the_fixed_capacity_are_rejected():
    import torch
    from paper_2605_13766_gb300 import RodError
    from paper_2605_13766_gb300.binding import contact_forces_noalloc
    n_rods, n = 1100, 128                      # 140,800 elements > 131,072
    node_off = torch.arange(0, (n + 1) * (n_rods + 1), n + 1, dtype=torch.int32, device="cuda")
    radius = torch.full((n_rods,), 0.004, dtype=torch.float64, device="cuda")
    N = (n + 1) * n_rods
    x = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(x)
    with pytest.raises(RodError) as ei:
        contact_forces_noalloc(node_off, radius, x, x, 1e4, 10.0, 0.0, f)
    assert ei.value.status == -5
    assert "capacity" in str(ei.value)
