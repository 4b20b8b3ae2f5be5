"""Rods longer than a thread block holds: stepped by a cooperative launch over the whole GPU with
the same stage code (working arrays in global memory, grid-wide barriers).  Parity with the
oracle at the step's bars, and bit-identity with the block path when a small launch shape
sends ordinary rods down the cooperative path."""
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


def _gpu(p, shape=None):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    if shape is not None:
        s.set_launch(*shape)
    s.set_state(*p.state())
    return s


def _mixed_long(seed=3):
    """Two long rods (1500 and 2600 elements, 2 mm each) between short ones, clamped and free,
    with actuation, muscle couples, a magnetic field and a wall."""
    from rodgen import _straight_rods
    rng = np.random.default_rng(seed)
    n_elem = np.array([40, 1500, 7, 2600, 64, 1], dtype=np.int32)
    R = n_elem.size
    rest = np.full(int(n_elem.sum()), 2e-3)
    base = rng.uniform(-0.5, 0.5, (R, 3))
    d3 = rng.normal(size=(R, 3))
    d3 /= np.linalg.norm(d3, axis=1, keepdims=True)
    ref = rng.normal(size=(R, 3))
    x, Q = _straight_rods(n_elem, rest, base, d3, ref)
    E = int(n_elem.sum())
    p = rodgen.RodProblem(
        name="mixed_long", n_elem=n_elem, rest_len=rest, radius=np.full(R, 0.004), youngs=np.full(R, 1e6),
        shear_mod=np.full(R, 1e6 / 1.5), density=np.full(R, 1000.0), x=x, v=np.zeros_like(x), Q=Q,
        w=np.zeros((3, E)), clamp_base=np.array([1, 1, 0, 0, 1, 0], dtype=np.int8),
        gravity=np.array([0.0, 0.0, -9.81]), nu_damp=0.05,
        act_amp=np.full(R, 1e-6), act_period=np.full(R, 0.3), act_phase=rng.uniform(0, 6.28, R),
        muscle_amp=np.full(R, 2e-6), muscle_period=np.full(R, 0.1), muscle_wavelength=np.full(R, 0.5),
        muscle_phase=rng.uniform(0, 6.28, R),
        magnetization=np.vstack([np.zeros(E), np.zeros(E), np.full(E, 0.5)]),
        field_b0=np.array([1e-3, 0.0, 0.0]), field_bs=np.array([0.0, 1e-3, 0.0]), field_omega=30.0,
        wall_point=np.zeros((1, 3)), wall_normal=np.array([[0.0, 0.0, 1.0]]), wall_k=100.0,
        wall_c=0.1, wall_mu=0.2, wall_vslip=1e-3, dt=1e-5)
    p = rodgen.perturbed(p, seed=seed, pos=0.02, vel=0.05, rot=0.02, omega=1.0)
    # a floor that the lowest nodes touch by up to 0.5 mm
    return p.replace(wall_point=np.array([[0.0, 0.0, p.x[2].min() - 0.004 + 5e-4]]))


def test_long_rods_rhs_matches_oracle():
    p = _mixed_long()
    t = 0.0123
    av_ref, aw_ref = Oracle(p).rhs(*p.state(), t=t)
    s = _gpu(p)
    # the two long rods run cooperatively; the four short ones share one listed pack
    assert s.pack_info() == (1, 1, 2)
    av, aw = (a.cpu().numpy() for a in s.rhs(t))
    assert _rel(av, av_ref) <= 1e-12, _rel(av, av_ref)
    assert _rel(aw, aw_ref) <= 1e-12, _rel(aw, aw_ref)


def test_long_rods_trajectory_1000_steps():
    p = _mixed_long(seed=4)
    dt = 1e-5
    ref = Oracle(p).step(*p.state(), dt=dt, n_steps=1000)
    s = _gpu(p)
    s.step(1000, dt)
    got = s.get_state()
    L_max = 2600 * 2e-3
    assert np.abs(got[0] - ref[0]).max() / L_max <= 1e-9, np.abs(got[0] - ref[0]).max() / L_max
    assert _rel(got[2], ref[2]) <= 1e-9


def test_cooperative_path_is_bit_identical_to_the_block_path():
    """With 64 elements per block every rod of a carpet of 50-element rods still fits a block;
    with 32 none does: the cooperative launches must give the same state bit for bit."""
    p = rodgen.perturbed(rodgen.cilia_carpet(side=3, n=50), seed=5, pos=0.01, vel=0.05, rot=0.02, omega=2.0)
    a = _gpu(p, (64, 64))
    b = _gpu(p, (32, 32))
    a.step(200, 1e-5)
    b.step(200, 1e-5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    ra = [t.cpu().numpy() for t in a.rhs(0.5)]
    rb = [t.cpu().numpy() for t in b.rhs(0.5)]
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)


def test_long_rods_with_contact():
    """A long rod lying through a cloud of short rods: contact forces and a trajectory through
    collisions, with the long rod on the cooperative path (binning epilogue included)."""
    rng = np.random.default_rng(9)
    base = rodgen.random_packing(n_rods=30, nmin=5, nmax=20, box=0.06, rest_len=2e-3, radius=0.004, seed=9,
                                 speed=0.5, dt=2e-6, margin=-5e-4)
    n_long = 1200
    xl = np.zeros((3, n_long + 1))
    xl[0] = np.linspace(-1.2, 1.2, n_long + 1)
    xl[1] = 0.009               # a line that touches three short rods by under 1 mm
    xl[2] = 0.047
    Ql = np.zeros((9, n_long))
    Ql[[1, 5, 6]] = 1.0          # d1 = y, d2 = z, d3 = x
    p = base.replace(
        n_elem=np.concatenate([base.n_elem, [n_long]]).astype(np.int32),
        rest_len=np.concatenate([base.rest_len, np.full(n_long, 2e-3)]),
        radius=np.concatenate([base.radius, [0.004]]), youngs=np.concatenate([base.youngs, [1e6]]),
        shear_mod=np.concatenate([base.shear_mod, [1e6 / 1.5]]), density=np.concatenate([base.density, [1000.0]]),
        x=np.concatenate([base.x, xl], axis=1), v=np.concatenate([base.v, rng.normal(0, 0.1, (3, n_long + 1))], axis=1),
        Q=np.concatenate([base.Q, Ql], axis=1), w=np.concatenate([base.w, np.zeros((3, n_long))], axis=1))
    o = Oracle(p, broad_phase=0)
    f_ref = o.contact_forces(p.x, p.v)
    s = _gpu(p)
    f = s.contact_forces().cpu().numpy()
    long_nodes = slice(p.n_nodes - n_long - 1, p.n_nodes)
    assert np.abs(f_ref[:, long_nodes]).max() > 0.1          # the long rod is in contact
    assert _rel(f, f_ref) <= 1e-12
    ref = Oracle(p).step(*p.state(), dt=2e-6, n_steps=300)
    s.step(300, 2e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() / 2.4 <= 1e-9
