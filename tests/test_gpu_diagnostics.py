"""GPU energy, frame and tip diagnostics (rod_system_diagnostics) against the oracle's energy.

Each component is pinned on its own: a state in which only that part of the energy is non-zero
(velocities only, angular velocities only, stretched rods with uniform frames, rods twisted about
their tangents, loads on rods at rest), compared per rod with the oracle's energy of that rod
alone; a general state then checks the sum per rod and the totals.  Bar: 1e-12 relative.
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _base(seed=21):
    """Straight rods at rest of ragged lengths (1..150 elements: one to five warp passes)."""
    p = rodgen.random_packing(n_rods=30, nmin=1, nmax=150, box=2.0, rest_len=4e-3, radius=0.004, seed=seed,
                              allow_overlap=True, speed=0.0)
    z = np.zeros
    return p.replace(contact=False, v=z((3, p.n_nodes)), w=z((3, p.n_elems)), gravity=z(3), tip_force=None)


def _one_rod(p, r):
    eo, no = p.elem_offsets(), p.node_offsets()
    e0, e1, n0, n1 = int(eo[r]), int(eo[r + 1]), int(no[r]), int(no[r + 1])
    n = e1 - e0

    def cut(a, lo, hi):
        return None if a is None else np.ascontiguousarray(a[:, lo:hi])

    return rodgen.RodProblem(
        name="one", n_elem=p.n_elem[r:r + 1].copy(), rest_len=p.rest_len[e0:e1].copy(),
        radius=p.radius[r:r + 1].copy(), youngs=p.youngs[r:r + 1].copy(), shear_mod=p.shear_mod[r:r + 1].copy(),
        density=p.density[r:r + 1].copy(), x=cut(p.x, n0, n1), v=cut(p.v, n0, n1), Q=cut(p.Q, e0, e1),
        w=cut(p.w, e0, e1), alpha_c=p.alpha_c,
        rest_kappa=cut(p.rest_kappa, e0 - r, e1 - r - 1) if n > 1 else None,
        rest_sigma=cut(p.rest_sigma, e0, e1), gravity=np.array(p.gravity, dtype=float),
        tip_force=cut(p.tip_force, r, r + 1))


def _oracle_per_rod(p):
    out = []
    for r in range(p.n_rods):
        q = _one_rod(p, r)
        out.append(Oracle(q).energy(*q.state()))
    return np.array(out)


def _gpu_rows(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    rows, tot = s.diagnostics()
    return rows.cpu().numpy(), tot, s


def _close(got, ref, scale=None):
    scale = np.abs(ref).max() if scale is None else scale
    assert np.abs(got - ref).max() <= TOL * scale, (np.abs(got - ref).max(), scale)


def test_translational_kinetic_energy():
    p = _base()
    rng = np.random.default_rng(1)
    p = p.replace(v=rng.normal(0, 0.3, (3, p.n_nodes)))
    rows, tot, _ = _gpu_rows(p)
    ref = _oracle_per_rod(p)
    _close(rows[0], ref)
    assert np.abs(rows[1]).max() == 0.0 and np.abs(rows[4]).max() == 0.0
    assert np.abs(rows[2] + rows[3]).max() <= 1e-20 * ref.max()   # straight rods at rest length


def test_rotational_kinetic_energy():
    p = _base()
    rng = np.random.default_rng(2)
    p = p.replace(w=rng.normal(0, 5.0, (3, p.n_elems)))
    rows, _, _ = _gpu_rows(p)
    _close(rows[1], _oracle_per_rod(p))
    assert np.abs(rows[0]).max() == 0.0


def test_shear_stretch_energy():
    """Nodes moved off the line while every element keeps its frame: sigma != 0, kappa = 0."""
    p = _base()
    rng = np.random.default_rng(3)
    x = p.x + rng.normal(0, 2e-4, p.x.shape)
    sig = rng.normal(0, 1e-3, (3, p.n_elems))
    p = p.replace(x=x, rest_sigma=sig)
    rows, _, _ = _gpu_rows(p)
    ref = _oracle_per_rod(p)
    _close(rows[2], ref)
    assert np.abs(rows[3]).max() <= 1e-20 * ref.max()


def test_bend_twist_energy():
    """Frames twisted about the tangent by a varying angle, with a rest curvature: kappa != 0,
    sigma = 0 (rounding only)."""
    p = _base()
    rng = np.random.default_rng(4)
    Q = p.Q.reshape(3, 3, -1).copy()
    phi = np.cumsum(rng.normal(0, 0.4, p.n_elems))   # up to a few radians between neighbours' sums
    c, s = np.cos(phi), np.sin(phi)
    d1, d2 = Q[0].copy(), Q[1].copy()
    Q[0] = c * d1 + s * d2
    Q[1] = -s * d1 + c * d2
    kap0 = rng.normal(0, 0.5, (3, p.n_voronoi))
    p = p.replace(Q=Q.reshape(9, -1), rest_kappa=kap0)
    rows, _, _ = _gpu_rows(p)
    ref = _oracle_per_rod(p)
    _close(rows[3], ref)
    assert np.abs(rows[2]).max() <= 1e-12 * ref.max()


def test_work_potential_of_gravity_and_tip_forces():
    p = _base()
    rng = np.random.default_rng(5)
    p = p.replace(gravity=np.array([0.3, -9.81, 1.2]), tip_force=rng.normal(0, 1e-2, (3, p.n_rods)))
    rows, _, _ = _gpu_rows(p)
    ref = _oracle_per_rod(p)
    _close(rows[4], ref)


def test_general_state_sums_and_totals():
    p = rodgen.perturbed(_base(), seed=6, pos=1e-3, vel=0.2, rot=0.3)
    rng = np.random.default_rng(6)
    p = p.replace(gravity=np.array([0.0, -9.81, 0.0]), tip_force=rng.normal(0, 1e-2, (3, p.n_rods)),
                  rest_kappa=rng.normal(0, 0.3, (3, p.n_voronoi)), rest_sigma=rng.normal(0, 1e-3, (3, p.n_elems)))
    rows, tot, s = _gpu_rows(p)
    per_rod = _oracle_per_rod(p)
    scale = np.abs(rows[:5]).sum(axis=0)
    assert np.all(np.abs(rows[:5].sum(axis=0) - per_rod) <= TOL * scale)
    H = Oracle(p).energy(*p.state())
    assert abs(tot[:5].sum() - H) <= TOL * scale.sum()
    assert np.all(np.abs(tot[:5] - rows[:5].sum(axis=1)) <= 1e-13 * np.abs(rows[:5]).sum(axis=1))
    # rows 6-8: the tip of every rod (its last node), copied bit for bit
    tips = p.x[:, p.node_offsets()[1:] - 1]
    assert np.array_equal(rows[6:9], tips)
    # the totals do not change between calls, and a call with totals launches two kernels
    n0 = s.launch_count
    _, tot2 = s.diagnostics(per_rod=False)
    assert np.array_equal(tot, tot2) and s.launch_count - n0 == 2


def test_orthonormality_row():
    """Directors pushed off orthonormal by 1e-9: row 5 is the oracle's entrywise max |Q Q^T - I|,
    per rod and overall.  (The bend energy of such frames is not compared: the rotation angle of
    a non-orthogonal relative rotation depends on the formula, atan2 of the antisymmetric part
    and the trace or the series in the antisymmetric part alone, at 1e-8 here.)"""
    p = rodgen.perturbed(_base(), seed=8, pos=1e-3, vel=0.2, rot=0.3)
    rng = np.random.default_rng(8)
    p = p.replace(Q=p.Q + rng.normal(0, 1e-9, p.Q.shape))
    rows, tot, _ = _gpu_rows(p)
    for r in range(p.n_rods):
        q = _one_rod(p, r)
        assert abs(rows[5, r] - Oracle(q).orthonormality_error(q.Q)) <= 1e-15
    assert tot[5] == rows[5].max() and abs(tot[5] - Oracle(p).orthonormality_error(p.Q)) <= 1e-15
    assert 1e-10 < tot[5] < 1e-7


def test_energy_after_steps_follows_the_oracle():
    """Undamped, unactuated carpet under gravity: the energy of the GPU state after 1000 steps against the
    oracle's energy of its own state after the same steps (positions agree to 1e-9)."""
    p = rodgen.perturbed(rodgen.cilia_carpet(side=3, n=50), seed=7, vel=0.05, rot=0.05)
    p = p.replace(nu_damp=0.0, stokes_gamma=0.0, gravity=np.array([0.0, 0.0, -9.81]), act_amp=None,
                  act_period=None, act_phase=None)
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    e0 = s.energy()
    s.step(1000, 1e-5)
    e1 = s.energy()
    o = Oracle(p)
    ref0 = o.energy(*p.state())
    ref_state = o.step(*p.state(), dt=1e-5, n_steps=1000)
    ref1 = o.energy(*ref_state)
    scale = abs(ref0) + abs(ref1)
    assert abs(e0 - ref0) <= TOL * scale
    assert abs(e1 - ref1) <= 1e-8 * scale
    # symplectic step without damping: the energy moves by far less than it holds
    assert abs(e1 - e0) <= 1e-2 * scale
