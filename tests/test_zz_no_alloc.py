"""The allocation-free contact entry point (rod_contact_forces_noalloc) against the system's own
contact forces (rod_system_contact_forces) and the oracle's exhaustive search on the same states,
plus the paths that size its fixed scratch: a grid that must grow to fit, finite but huge
coordinates, a cell that holds too many segments, non-finite positions.

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


def _oracle_forces(p):
    from oracle.oracle import Oracle
    return Oracle(p, broad_phase=0).contact_forces(p.x, p.v)


def test_two_calls_in_a_row_match_the_system_entry_point():
    first = _packing(21)
    second = rodgen.perturbed(_packing(22, n_rods=120, box=0.1), seed=3, pos=0.05, vel=0.5, rot=0.0, omega=0.0)
    for p in (first, second):
        ref = _system_forces(p)
        got = _noalloc_forces(p)
        scale = np.abs(ref).max()
        assert scale > 1.0                      # there is contact to compare
        assert np.abs(got - ref).max() <= TOL * scale
        orc = _oracle_forces(p)
        assert np.abs(got - orc).max() <= TOL * np.abs(orc).max()


def _two_clusters(offset, n_second=25):
    """Two contact-rich clusters of 25 rods (the second cut to its first n_second rods), the
    second moved by `offset` (m) along each axis."""
    a = rodgen.random_packing(n_rods=25, nmin=3, nmax=20, box=0.06, rest_len=2e-3, radius=0.004, seed=31,
                              allow_overlap=True, speed=0.3)
    b = rodgen.random_packing(n_rods=25, nmin=3, nmax=20, box=0.06, rest_len=2e-3, radius=0.004, seed=32,
                              allow_overlap=True, speed=0.3).take_rods(0, n_second)
    cat = lambda u, w: np.concatenate([u, w], axis=-1)
    return a.replace(n_elem=cat(a.n_elem, b.n_elem), rest_len=cat(a.rest_len, b.rest_len),
                     radius=cat(a.radius, b.radius), youngs=cat(a.youngs, b.youngs),
                     shear_mod=cat(a.shear_mod, b.shear_mod), density=cat(a.density, b.density),
                     x=cat(a.x, b.x + offset), v=cat(a.v, b.v), Q=cat(a.Q, b.Q), w=cat(a.w, b.w))


def test_grid_that_must_grow_to_fit_the_scratch():
    # 100 m between the clusters with 1 cm cells would need ~10^12 cells: the cell edge grows
    # until the grid fits ROD_NOALLOC_MAX_CELLS, and the search stays exact
    p = _two_clusters(100.0)
    orc = _oracle_forces(p)
    assert np.abs(orc).max() > 1.0
    for _ in range(2):
        got = _noalloc_forces(p)
        assert np.abs(got - orc).max() <= TOL * np.abs(orc).max()
    sysf = _system_forces(p)
    assert np.abs(got - sysf).max() <= TOL * np.abs(sysf).max()


def test_finite_but_huge_coordinates_give_exact_forces():
    # one rod moved to 1e30 m (its nodes coincide there in FP64): the grid's dimensions are
    # clamped before any integer conversion and the cell edge jumps to the extent / 63
    p = _two_clusters(1e30, n_second=1)
    orc = _oracle_forces(p)
    got = _noalloc_forces(p)
    assert np.abs(orc).max() > 1.0
    assert np.abs(got - orc).max() <= TOL * np.abs(orc).max()


def _one_element_rods(n_rods, centre_spread, seed=5):
    p = rodgen.random_packing(n_rods=n_rods, nmin=1, nmax=1, box=centre_spread, rest_len=1e-4, radius=0.004,
                              seed=seed, allow_overlap=True, speed=0.1)
    return p


def test_a_cell_with_more_than_512_segments_is_rejected():
    from paper_2605_13766_gb300 import RodError
    p = _one_element_rods(600, 1e-3)            # 600 segments in one cell of edge >= 8 mm
    with pytest.raises(RodError) as ei:
        _noalloc_forces(p)
    assert ei.value.status == -5 and "512" in str(ei.value)
    # the next call on a fine state is unaffected by the rejected one
    q = _packing(23)
    ref = _system_forces(q)
    assert np.abs(_noalloc_forces(q) - ref).max() <= TOL * np.abs(ref).max()


def test_non_finite_positions_are_rejected():
    from paper_2605_13766_gb300 import RodError
    p = _packing(24)
    x = p.x.copy()
    x[1, 7] = np.nan
    with pytest.raises(RodError) as ei:
        _noalloc_forces(p.replace(x=x))
    assert ei.value.status == -3


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
