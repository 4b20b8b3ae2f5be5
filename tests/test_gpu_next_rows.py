"""GPU parity of the rows after the step against the CPU oracle: the magnetic couple (Eq. 2)
with a rotating field, travelling-wave muscle couples, rod-wall contact with friction and
rod-rod friction.  Same bars as the step: right-hand sides to 1e-12 (max-norm relative per
array), positions to 1e-9 of the system size after 1000 steps (400 with contact)."""
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


def _gpu(p):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    return s


def _magnetic_muscle_carpet(side=4, n=50, seed=21):
    """Clamped carpet, magnetized along d3 in a rotating field, with muscle waves and a floor
    wall plus a slanted side wall, perturbed so that every term acts."""
    rng = np.random.default_rng(seed)
    p = rodgen.cilia_carpet(side=side, n=n, seed=seed)
    R, E = p.n_rods, p.n_elems
    mag = np.zeros((3, E))
    mag[2] = rng.uniform(0.5, 1.5, E)
    mag[0] = rng.normal(0, 0.1, E)
    # the side wall only touches the base of the rods of the last column (x = 0.05 (side - 1))
    walls_p = np.array([[0.0, 0.0, 0.0], [0.05 * (side - 1) + 0.005, 0.0, 0.0]])
    nrm = np.array([[0.0, 0.0, 1.0], [-1.0, 0.2, 0.1]])
    nrm[1] /= np.linalg.norm(nrm[1])
    q = p.replace(magnetization=mag, field_b0=np.array([0.0, 0.0, 2e-3]), field_bc=np.array([5e-3, 0.0, 0.0]),
                  field_bs=np.array([0.0, 5e-3, 0.0]), field_omega=2 * np.pi * 3.0,
                  muscle_amp=rng.uniform(1e-5, 5e-5, R), muscle_period=rng.uniform(0.2, 1.0, R),
                  muscle_wavelength=rng.uniform(0.1, 0.4, R), muscle_phase=rng.uniform(0, 6.28, R),
                  wall_point=walls_p, wall_normal=nrm, wall_velocity=np.array([[0.0, 0.0, 0.0], [-0.01, 0.0, 0.0]]),
                  wall_k=200.0, wall_c=0.5, wall_mu=0.3, wall_vslip=1e-4)
    q = rodgen.perturbed(q, seed=seed, pos=0.02, vel=0.05, rot=0.03, omega=2.0)
    # pull the base layer into the floor so the floor wall acts on the first nodes
    q.x[2] -= 0.004
    return q


def test_rhs_with_magnetic_muscle_and_walls_matches_oracle():
    p = _magnetic_muscle_carpet()
    o = Oracle(p)
    t = 0.0731
    av_ref, aw_ref = o.rhs(*p.state(), t=t)
    # every term acts: compare with the same system without each of them
    for drop in ({"magnetization": None}, {"muscle_amp": None}, {"wall_point": None, "wall_normal": None}):
        av0, aw0 = Oracle(p.replace(**drop)).rhs(*p.state(), t=t)
        assert max(_rel(av0, av_ref), _rel(aw0, aw_ref)) > 1e-6, drop
    av, aw = (a.cpu().numpy() for a in _gpu(p).rhs(t))
    assert _rel(av, av_ref) <= 1e-12, _rel(av, av_ref)
    assert _rel(aw, aw_ref) <= 1e-12, _rel(aw, aw_ref)


def test_trajectory_with_magnetic_muscle_and_walls_1000_steps():
    p = _magnetic_muscle_carpet(side=3)
    dt = 1e-5
    ref = Oracle(p).step(*p.state(), dt=dt, n_steps=1000)
    s = _gpu(p)
    s.step(1000, dt)
    got = s.get_state()
    size = 0.2
    assert np.abs(got[0] - ref[0]).max() / size <= 1e-9, np.abs(got[0] - ref[0]).max() / size
    assert _rel(got[2], ref[2]) <= 1e-9


def _dense_with_friction(n_rods=80, box=0.08, seed=1, mu=0.4):
    p = rodgen.random_packing(n_rods=n_rods, nmin=3, nmax=30, box=box, rest_len=2e-3, radius=0.004,
                              seed=seed, allow_overlap=True, speed=0.3)
    return p.replace(contact_mu=mu, contact_vslip=1e-3)


@pytest.mark.parametrize("seed", [1, 2])
def test_contact_forces_with_friction_match_exhaustive_oracle(seed):
    p = _dense_with_friction(seed=seed)
    ref = Oracle(p, broad_phase=0).contact_forces(p.x, p.v)
    ref0 = Oracle(p.replace(contact_mu=0.0), broad_phase=0).contact_forces(p.x, p.v)
    assert _rel(ref0, ref) > 1e-3                      # friction changes the forces
    got = _gpu(p).contact_forces().cpu().numpy()
    assert _rel(got, ref) <= 1e-12, _rel(got, ref)
    assert np.abs(got.sum(1)).max() <= 1e-11 * np.abs(ref).max()


def test_trajectory_with_friction_and_a_box_400_steps():
    """Rods pressed into each other inside a box of six walls, with rod-rod and wall friction."""
    box = 0.08
    p = rodgen.random_packing(n_rods=40, nmin=8, nmax=40, box=box, rest_len=2e-3, radius=0.004, seed=6,
                              speed=1.0, dt=2e-6, margin=-1e-3)
    # walls just inside the extreme nodes' spheres: a few nodes touch them by up to 0.5 mm
    lo = p.x.min(axis=1) - 0.004 + 5e-4
    hi = p.x.max(axis=1) + 0.004 - 5e-4
    pts = np.array([lo, hi, lo, hi, lo, hi], dtype=float)
    nrm = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=float)
    p = p.replace(contact_mu=0.3, contact_vslip=1e-3, wall_point=pts, wall_normal=nrm, wall_k=1e4,
                  wall_c=5.0, wall_mu=0.2, wall_vslip=1e-3, gravity=np.array([0.0, 0.0, -9.81]))
    o = Oracle(p)
    assert np.abs(o.contact_forces(p.x, p.v)).max() > 0.5
    av, _ = o.rhs(*p.state())
    av0, _ = Oracle(p.replace(wall_point=None, wall_normal=None)).rhs(*p.state())
    assert _rel(av0, av) > 1e-6                          # the walls act
    ref = o.step(*p.state(), dt=2e-6, n_steps=400)
    s = _gpu(p)
    s.step(400, 2e-6)
    got = s.get_state()
    size = float((hi - lo).max())
    assert np.abs(got[0] - ref[0]).max() / size <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7


def test_adjoint_refuses_rod_rod_contact_only():
    from paper_2605_13766_gb300 import RodError
    p = _magnetic_muscle_carpet(side=2)
    s = _gpu(p)
    s.forward_checkpointed(10, 1e-5, 5)          # magnetic couple, muscles and walls: covered
    q = _dense_with_friction(n_rods=10, box=0.05)
    s = _gpu(q)
    with pytest.raises(RodError):
        s.forward_checkpointed(10, 1e-5, 5)


def test_invalid_walls_and_friction_are_rejected():
    from paper_2605_13766_gb300 import RodError
    p = _magnetic_muscle_carpet(side=2)
    bad = p.wall_normal.copy()
    bad[0] *= 2.0
    with pytest.raises(RodError):
        _gpu(p.replace(wall_normal=bad))
    s = _gpu(p)
    with pytest.raises(RodError):
        s.friction(0.3, 0.0)
    with pytest.raises(RodError):
        s.friction(-0.1, 1e-3)
