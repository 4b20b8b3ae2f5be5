"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bars (spec tolerances, norms fixed in the design notes):
  * right-hand side: |a_gpu - a_ref|_inf / |a_ref|_inf <= 1e-12 for node and element arrays;
  * trajectories: |x_gpu - x_ref|_inf / L_max <= 1e-9 after 1000 steps.
The GPU evaluates the same definitions in a different rounding order (FMA contraction,
series evaluation of the rotation exponential/logarithm, precomputed reciprocals).
"""
import numpy as np
import pytest

import rodgen
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-12
POS_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


def _gpu(p, shape=None):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    if shape is not None:
        s.set_launch(*shape)
    s.set_state(*p.state())
    return s


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _mixed_rods(n_rods=24, nmin=1, nmax=70, seed=3, clamp_every=3):
    """Free and clamped rods of ragged lengths (1..nmax elements), several thread blocks."""
    rng = np.random.default_rng(seed)
    p = rodgen.random_packing(n_rods=n_rods, nmin=nmin, nmax=nmax, box=2.0, rest_len=4e-3, radius=0.004,
                              seed=seed, allow_overlap=True, speed=0.2)
    clamp = np.zeros(n_rods, dtype=np.int8)
    clamp[::clamp_every] = 1
    return p.replace(contact=False, clamp_base=clamp, gravity=np.array([0.0, -1.0, -9.81]), nu_damp=0.05,
                     stokes_gamma=0.02, tip_force=rng.normal(0, 1e-3, (3, n_rods)),
                     rest_sigma=rng.normal(0, 1e-3, (3, p.n_elems)),
                     elem_couple=rng.normal(0, 1e-6, (3, p.n_elems)),
                     rest_kappa=rng.normal(0, 0.5, (3, p.n_voronoi)),
                     act_amp=np.full(n_rods, 1e-6), act_period=np.full(n_rods, 0.5),
                     act_phase=rng.uniform(0, 6.28, n_rods))


def _rhs_cases():
    yield "cantilever", rodgen.perturbed(rodgen.cantilever(), seed=1)
    yield "carpet", rodgen.perturbed(rodgen.cilia_carpet(side=4, n=50), seed=2, rot=0.02)
    yield "adjoint", rodgen.perturbed(rodgen.adjoint_batch(n_rods=8, n=64), seed=3)
    yield "mixed", rodgen.perturbed(_mixed_rods(), seed=4, pos=0.01, rot=0.05)


@pytest.mark.parametrize("name,p", list(_rhs_cases()), ids=[c[0] for c in _rhs_cases()])
def test_rhs_matches_oracle(name, p):
    o = Oracle(p)
    t = 0.123
    av_ref, aw_ref = o.rhs(*p.state(), t=t)
    s = _gpu(p)
    av, aw = s.rhs(t)
    av, aw = av.cpu().numpy(), aw.cpu().numpy()
    assert _rel(av, av_ref) <= RHS_TOL, _rel(av, av_ref)
    assert _rel(aw, aw_ref) <= RHS_TOL, _rel(aw, aw_ref)


@pytest.mark.parametrize("shape", [(128, 64), (256, 128), (384, 256), (512, 512), (768, 256)])
def test_rhs_independent_of_launch_shape(shape):
    p = rodgen.perturbed(_mixed_rods(n_rods=40, nmax=100, seed=9), seed=5)
    if shape[0] < 100:
        pytest.skip("shape cannot hold the longest rod")
    o = Oracle(p)
    av_ref, aw_ref = o.rhs(*p.state(), t=0.0)
    s = _gpu(p, shape)
    av, aw = (a.cpu().numpy() for a in s.rhs(0.0))
    assert _rel(av, av_ref) <= RHS_TOL and _rel(aw, aw_ref) <= RHS_TOL


def _traj(p, steps, dt, shape=None, chunks=(None,)):
    o = Oracle(p)
    ref = o.step(*p.state(), dt=dt, n_steps=steps)
    s = _gpu(p, shape)
    if chunks == (None,):
        s.step(steps, dt)
    else:
        for c in chunks:
            s.step(c, dt)
    got = s.get_state()
    return ref, got


@pytest.mark.parametrize("name,p,dt", [
    ("cantilever", rodgen.cantilever(), 1e-5),
    ("carpet", rodgen.cilia_carpet(side=4, n=50), 1e-5),
    ("adjoint", rodgen.adjoint_batch(n_rods=8, n=64), 1e-5),
    ("mixed", _mixed_rods(), 2e-6),
], ids=["cantilever", "carpet", "adjoint", "mixed"])
def test_trajectory_1000_steps(name, p, dt):
    ref, got = _traj(p, 1000, dt)
    L = max(p.rest_len[p.elem_offsets()[r]:p.elem_offsets()[r + 1]].sum() for r in range(p.n_rods))
    assert np.abs(got[0] - ref[0]).max() / L <= POS_TOL
    for a, b in zip(got[1:], ref[1:]):
        assert np.all(np.isfinite(a))
    # velocities / directors / angular velocities agree to the same relative order
    assert _rel(got[2], ref[2]) <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7


def test_listed_packs_match_the_oracle():
    """Rods of mixed lengths at 256 node slots per block: best fit needs fewer packs than
    packing in index order, so the packs list rods that are not consecutive.  The right-hand
    side and a 1000-step trajectory stay at the oracle's bars.  Equal rods keep consecutive packs."""
    p = _mixed_rods()
    s = _gpu(p, (256, 128))
    n_packs, n_listed, n_long = s.pack_info()
    assert n_listed > 0 and n_long == 0
    pr = rodgen.perturbed(p, seed=4, pos=0.01, rot=0.05)
    av_ref, aw_ref = Oracle(pr).rhs(*pr.state(), t=0.05)
    av, aw = (a.cpu().numpy() for a in _gpu(pr, (256, 128)).rhs(0.05))
    assert _rel(av, av_ref) <= RHS_TOL and _rel(aw, aw_ref) <= RHS_TOL
    ref, got = _traj(p, 1000, 2e-6, shape=(256, 128))
    L = max(p.rest_len[p.elem_offsets()[r]:p.elem_offsets()[r + 1]].sum() for r in range(p.n_rods))
    assert np.abs(got[0] - ref[0]).max() / L <= POS_TOL
    assert _rel(got[2], ref[2]) <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7
    c = _gpu(rodgen.cilia_carpet(side=4, n=50), (384, 192))
    assert c.pack_info()[1] == 0


def test_chunked_steps_equal_one_call():
    p = rodgen.perturbed(rodgen.cilia_carpet(side=3, n=50), seed=8)
    s1 = _gpu(p)
    s1.step(300, 1e-5)
    a = s1.get_state()
    s2 = _gpu(p)
    for _ in range(3):
        s2.step(100, 1e-5)
    b = s2.get_state()
    # the fused kinematic update differs from split halves only by rounding
    assert np.abs(a[0] - b[0]).max() < 1e-13
    assert abs(s2.time - 300 * 1e-5) < 1e-15


def test_single_element_rods_and_capacity_edge():
    n_elem = np.array([1, 1, 2, 384, 1, 3, 383, 1], dtype=np.int32)
    base = _mixed_rods(n_rods=8, seed=11)
    rl = np.full(int(n_elem.sum()), 2e-3)
    p = rodgen.random_packing(n_rods=8, nmin=1, nmax=2, seed=11, allow_overlap=True, rest_len=2e-3)
    # rebuild straight rods with the exact lengths above
    x, v, Q, w = _straight(n_elem, rl, seed=11)
    q = p.replace(n_elem=n_elem, rest_len=rl, x=x, v=v, Q=Q, w=w, contact=False,
                  clamp_base=np.array([1, 0, 1, 0, 0, 1, 1, 0], dtype=np.int8), gravity=np.array([0, 0, -9.81]))
    q = rodgen.perturbed(q, seed=12, pos=0.01, rot=0.05)
    o = Oracle(q)
    av_ref, aw_ref = o.rhs(*q.state())
    s = _gpu(q, (384, 128))
    av, aw = (a.cpu().numpy() for a in s.rhs(0.0))
    assert _rel(av, av_ref) <= RHS_TOL and _rel(aw, aw_ref) <= RHS_TOL
    ref = o.step(*q.state(), dt=1e-6, n_steps=200)
    s.step(200, 1e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() <= 1e-12


def _straight(n_elem, rl, seed):
    rng = np.random.default_rng(seed)
    R = len(n_elem)
    E = int(n_elem.sum())
    x = np.zeros((3, E + R))
    Q = np.zeros((9, E))
    e0 = n0 = 0
    for r in range(R):
        d3 = rng.normal(size=3)
        d3 /= np.linalg.norm(d3)
        d1 = np.cross(d3, [0.3, 0.5, 0.8])
        d1 /= np.linalg.norm(d1)
        d2 = np.cross(d3, d1)
        base = rng.uniform(0, 1, 3)
        s = np.concatenate([[0], np.cumsum(rl[e0:e0 + n_elem[r]])])
        x[:, n0:n0 + n_elem[r] + 1] = base[:, None] + d3[:, None] * s[None, :]
        Q[:, e0:e0 + n_elem[r]] = np.concatenate([d1, d2, d3])[:, None]
        e0 += n_elem[r]
        n0 += n_elem[r] + 1
    return x, np.zeros_like(x), Q, np.zeros((3, E))


def test_orthonormality_after_10k_steps():
    p = rodgen.perturbed(rodgen.cilia_carpet(side=4, n=50), seed=13, rot=0.05, omega=20.0)
    s = _gpu(p)
    s.step(10_000, 1e-5)
    Q = s.get_state()[2]
    M = Q.T.reshape(-1, 3, 3)
    err = np.abs(M @ M.transpose(0, 2, 1) - np.eye(3)).max()
    assert err < 1e-12
    assert np.all(np.linalg.det(M) > 0)


def test_full_carpet_sampled_rods():
    """Full 64 x 64 x 50 carpet on the GPU for 200 steps; rods are independent without contact,
    so the oracle advances a sample of rods on their own and they must match."""
    p = rodgen.cilia_carpet()
    s = _gpu(p)
    s.step(200, 1e-5)
    got = s.get_state()
    noff, eoff = p.node_offsets(), p.elem_offsets()
    for r in (0, 1, 777, 2048, 4095):
        sub = _subset(p, [r])
        ref = Oracle(sub).step(*sub.state(), dt=1e-5, n_steps=200)
        xs = got[0][:, noff[r]:noff[r + 1]]
        assert np.abs(xs - ref[0]).max() / 0.2 <= POS_TOL
        assert np.abs(got[2][:, eoff[r]:eoff[r + 1]] - ref[2]).max() <= 1e-10


def _subset(p, rods):
    noff, eoff = p.node_offsets(), p.elem_offsets()
    voff = eoff - np.arange(len(eoff))
    nsl = np.concatenate([np.arange(noff[r], noff[r + 1]) for r in rods])
    esl = np.concatenate([np.arange(eoff[r], eoff[r + 1]) for r in rods])
    vsl = np.concatenate([np.arange(voff[r], voff[r + 1]) for r in rods])
    pick = lambda a: None if a is None else a[..., rods]
    return p.replace(
        n_elem=p.n_elem[rods], rest_len=p.rest_len[esl], radius=p.radius[rods], youngs=p.youngs[rods],
        shear_mod=p.shear_mod[rods], density=p.density[rods], x=p.x[:, nsl], v=p.v[:, nsl], Q=p.Q[:, esl],
        w=p.w[:, esl], clamp_base=pick(p.clamp_base),
        rest_kappa=None if p.rest_kappa is None else p.rest_kappa[:, vsl],
        rest_sigma=None if p.rest_sigma is None else p.rest_sigma[:, esl],
        elem_couple=None if p.elem_couple is None else p.elem_couple[:, esl],
        tip_force=None if p.tip_force is None else p.tip_force[:, rods],
        act_amp=pick(p.act_amp), act_period=pick(p.act_period), act_phase=pick(p.act_phase))


def test_nonfinite_state_is_reported_and_cleared():
    import torch
    from paper_2605_13766_gb300 import RodError
    p = rodgen.cantilever(n=20)
    s = _gpu(p)
    x, v, Q, w = (torch.tensor(a, device="cuda") for a in p.state())
    v[1, 5] = float("nan")
    s.set_state(x, v, Q, w)
    with pytest.raises(RodError) as ei:
        s.step(10, 1e-5)
    assert ei.value.status == -3
    s.set_state(*p.state())
    s.step(10, 1e-5)
    # a host state with NaN/Inf is rejected (checked on the device after the copy) and leaves
    # the system without a state until the next good one
    for bad in ("x", "Q", "w"):
        arrs = dict(x=p.x, v=p.v, Q=p.Q, w=p.w)
        arrs[bad] = arrs[bad].copy()
        arrs[bad].flat[7] = np.inf if bad == "Q" else np.nan
        with pytest.raises(RodError) as ei:
            s.set_state(arrs["x"], arrs["v"], arrs["Q"], arrs["w"])
        assert ei.value.status == -1
        with pytest.raises(RodError) as ei:
            s.step(1, 1e-5)
        assert ei.value.status == -6
    s.set_state(*p.state())
    s.step(10, 1e-5)
    out = [np.full(a.shape, np.nan) for a in p.state()]
    got = s.get_state(out=out)
    assert all(g is o for g, o in zip(got, out)) and np.isfinite(out[0]).all()


def test_invalid_descriptions_are_rejected():
    from paper_2605_13766_gb300 import RodError, RodSystem
    p = rodgen.cantilever(n=10)
    with pytest.raises(RodError):
        RodSystem(p.replace(rest_len=-p.rest_len))
    with pytest.raises(RodError):
        RodSystem(p.replace(n_elem=np.array([0], dtype=np.int32), rest_len=np.zeros(0)))
    # a rod longer than a block holds is accepted (it takes the cooperative path)
    RodSystem(p.replace(n_elem=np.array([2000], dtype=np.int32), rest_len=np.full(2000, 1e-3)))
    s = RodSystem(p)
    with pytest.raises(RodError):
        s.step(1, 1e-5)          # no state yet
    s.set_state(*p.state())
    with pytest.raises(RodError):
        s.step(1, -1.0)
    with pytest.raises(RodError):
        s.set_launch(100, 0)     # not a multiple of 32


def test_cantilever_settles_to_the_oracles_elastica_state():
    """The cantilever workload's rod (1 m, r = 1 cm, E = 1 MPa, tip force 1e-2 N, far outside
    linear theory) at n = 25, critically damped and run for 252,000 steps of 1e-4 s to rest: the
    GPU's settled tip equals the oracle's to 1e-9 of the length, and both sit at the oracle
    pin's first-order distance below the nonlinear elastica's 0.3651 m."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "statics", os.path.join(os.path.dirname(os.path.abspath(__file__)), "test_oracle_statics.py"))
    statics = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(statics)
    L, r, F, n = 1.0, 0.01, 1e-2, 25
    A, I, EA, EI, GAs = statics._consts(r)
    w1 = 3.516 * np.sqrt(EI / (1000 * A * L ** 4))
    nu = 2 * 1000 * A * w1
    dt = min(1e-4, 0.1 * (L / n) / np.sqrt(1e6 / 1000))
    steps = int(14 / w1 / dt)
    p = rodgen.cantilever(n=n, length=L, radius=r, tip_force=F, nu=nu, dt=dt)
    xo = Oracle(p).step(*p.state(), dt=dt, n_steps=steps)[0]
    s = _gpu(p)
    s.step(steps, dt)
    xg, vg = s.get_state()[:2]
    assert np.abs(xg - xo).max() / L <= POS_TOL
    assert np.abs(vg).max() < 1e-5
    y_ref, _ = statics._elastica_tip(L, EI, F)
    assert -0.07 < xg[1, -1] / y_ref - 1 < -0.03
