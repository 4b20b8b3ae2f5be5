"""Skin-list contact search (rod_system_contact_skin) on the GPU.

A list built from the cell grid keeps, per segment, the other-rod segments within
r_a + r_b + skin; it is rebuilt on the device once a node has moved by skin / 2 since the
build.  Checked against the oracle (trajectories through several rebuilds, with friction, with
rods longer than a block, with segments whose candidates overflow the list) and against the
direct per-step search of the same library.
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


def _touching(n_rods, box, seed, nmin=8, nmax=40, speed=1.0):
    """Rods placed without deep overlap (at most 1 mm) so that contact acts from the first step."""
    return rodgen.random_packing(n_rods=n_rods, nmin=nmin, nmax=nmax, box=box, rest_len=2e-3, radius=0.004,
                                 seed=seed, speed=speed, dt=2e-6, margin=-1e-3)


def _gpu(p, skin, graphs=True):
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.contact_skin(skin)
    if not graphs:
        s.use_graphs(False)
    s.set_state(*p.state())
    return s


def test_trajectory_through_several_rebuilds_matches_oracle():
    """400 steps of 2 us at up to ~1.7 m/s move nodes by ~1.4 mm: a 0.2 mm skin is rebuilt
    several times on the way."""
    p = _touching(40, 0.08, 6)
    o = Oracle(p)
    assert np.abs(o.contact_forces(p.x, p.v)).max() > 0.5
    ref = o.step(*p.state(), dt=2e-6, n_steps=400)
    s = _gpu(p, 2e-4)
    s.step(400, 2e-6)
    got = s.get_state()
    assert s.contact_list_builds() >= 3
    assert np.abs(got[0] - ref[0]).max() / 0.08 <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7


@pytest.mark.parametrize("skin", [1e-9, 5e-4, 2e-2])
def test_skin_list_equals_the_direct_search(skin):
    """From a list rebuilt at every step (tiny skin) to one never rebuilt (a skin wider than
    the motion): the trajectory of the direct per-step search up to the order of summation."""
    p = _touching(200, 0.2, 12, nmin=16, nmax=64)
    n = 300
    a = _gpu(p, 0.0)
    a.step(n, 2e-6)
    b = _gpu(p, skin)
    b.step(n, 2e-6)
    builds = b.contact_list_builds()
    if skin == 1e-9:
        assert builds == n
    if skin == 2e-2:
        assert builds == 1
    ga, gb = a.get_state(), b.get_state()
    assert np.abs(ga[0] - gb[0]).max() / 0.2 <= 1e-12
    assert _rel(gb[1], ga[1]) <= 1e-9


def _bundle(n_side=3, gap=2e-4, rest_len=1e-3, radius=5e-3, n=24, tilt=0.02):
    """Rods on a square lattice at centre distance 2 r + gap, each tilted from the common axis by
    `tilt` in a random direction (exactly parallel segments have no unique closest points, and
    rounding would pick the force split), with elements much shorter than the radius: with a
    3 mm skin a segment has more than the list's 32 candidates within 2 r + skin."""
    from rodgen import _straight_rods
    rng = np.random.default_rng(3)
    R = n_side * n_side
    n_elem = np.full(R, n, dtype=np.int32)
    rest = np.full(R * n, rest_len)
    ij = np.array([(i, j) for i in range(n_side) for j in range(n_side)], dtype=float)
    base = np.zeros((R, 3))
    base[:, 0] = ij[:, 0] * (2 * radius + gap)
    base[:, 1] = ij[:, 1] * (2 * radius + gap)
    base[:, 2] = np.linspace(0.0, 3e-3, R)           # staggered along the axis
    phi = rng.uniform(0, 2 * np.pi, R)
    d3 = np.stack([tilt * np.cos(phi), tilt * np.sin(phi), np.ones(R)], axis=1)
    d3 /= np.linalg.norm(d3, axis=1, keepdims=True)
    ref = np.tile([1.0, 0.0, 0.0], (R, 1))
    x, Q = _straight_rods(n_elem, rest, base, d3, ref)
    E = int(n_elem.sum())
    p = rodgen.RodProblem(
        name="bundle", n_elem=n_elem, rest_len=rest, radius=np.full(R, radius), youngs=np.full(R, 1e6),
        shear_mod=np.full(R, 1e6 / 1.5), density=np.full(R, 1000.0), x=x,
        v=np.repeat(rng.uniform(-0.2, 0.2, (R, 3)), n + 1, axis=0).T.copy(), Q=Q, w=np.zeros((3, E)),
        clamp_base=np.zeros(R, dtype=np.int8), gravity=np.zeros(3), nu_damp=0.0, contact=True,
        contact_k=1e4, contact_c=10.0, dt=2e-6)
    return p


def test_overflowing_lists_scan_their_neighbourhood():
    skin = 3e-3
    p = _bundle()
    # brute force on the CPU: some segment has more other-rod segments within 2 r + skin than a
    # list holds (32), so the overflow scan runs
    off = p.node_offsets()
    rod = np.repeat(np.arange(p.n_rods), p.n_elem)
    nodes = np.concatenate([np.arange(off[r], off[r + 1] - 1) for r in range(p.n_rods)])
    mid = 0.5 * (p.x[:, nodes] + p.x[:, nodes + 1])
    d = np.linalg.norm(mid[:, :, None] - mid[:, None, :], axis=0)
    # segment distance <= midpoint distance: these pairs are all list candidates
    near = (d < 2 * 5e-3 + skin) & (rod[:, None] != rod[None, :])
    assert near.sum(1).max() > 32
    o = Oracle(p)
    assert np.abs(o.contact_forces(p.x, p.v)).max() > 0.5
    ref = o.step(*p.state(), dt=2e-6, n_steps=200)
    s = _gpu(p, skin)
    s.step(200, 2e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() / 0.024 <= 1e-9
    a = _gpu(p, 0.0)
    a.step(200, 2e-6)
    assert np.abs(a.get_state()[0] - got[0]).max() / 0.024 <= 1e-12


def test_friction_with_skin_list_matches_oracle():
    p = _touching(40, 0.08, 16).replace(contact_mu=0.4, contact_vslip=1e-3)
    ref = Oracle(p).step(*p.state(), dt=2e-6, n_steps=300)
    s = _gpu(p, 3e-4)
    s.friction(0.4, 1e-3)
    s.step(300, 2e-6)
    got = s.get_state()
    assert np.abs(got[0] - ref[0]).max() / 0.08 <= 1e-9
    assert _rel(got[1], ref[1]) <= 1e-7


def test_long_rod_through_a_cloud_with_skin_list():
    """A 1200-element rod (cooperative launches) through short rods: the displacement of the
    long rod is tracked by the grid-wide path."""
    rng = np.random.default_rng(9)
    base = rodgen.random_packing(n_rods=30, nmin=5, nmax=20, box=0.06, rest_len=2e-3, radius=0.004, seed=9,
                                 speed=0.5, dt=2e-6, margin=-5e-4)
    n_long = 1200
    xl = np.zeros((3, n_long + 1))
    xl[0] = np.linspace(-1.2, 1.2, n_long + 1)
    xl[1] = 0.009
    xl[2] = 0.047
    Ql = np.zeros((9, n_long))
    Ql[[1, 5, 6]] = 1.0
    p = base.replace(
        n_elem=np.concatenate([base.n_elem, [n_long]]).astype(np.int32),
        rest_len=np.concatenate([base.rest_len, np.full(n_long, 2e-3)]),
        radius=np.concatenate([base.radius, [0.004]]), youngs=np.concatenate([base.youngs, [1e6]]),
        shear_mod=np.concatenate([base.shear_mod, [1e6 / 1.5]]), density=np.concatenate([base.density, [1000.0]]),
        x=np.concatenate([base.x, xl], axis=1), v=np.concatenate([base.v, rng.normal(0, 0.1, (3, n_long + 1))], axis=1),
        Q=np.concatenate([base.Q, Ql], axis=1), w=np.concatenate([base.w, np.zeros((3, n_long))], axis=1))
    ref = Oracle(p).step(*p.state(), dt=2e-6, n_steps=300)
    s = _gpu(p, 2e-5)
    s.step(300, 2e-6)
    got = s.get_state()
    assert s.contact_list_builds() >= 2
    assert np.abs(got[0] - ref[0]).max() / 2.4 <= 1e-9


def test_graph_replay_equals_eager_with_skin_list():
    p = _touching(60, 0.1, 14)
    a = _gpu(p, 2e-4)
    a.step(100, 2e-6)
    b = _gpu(p, 2e-4, graphs=False)
    b.step(100, 2e-6)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.contact_list_builds() == b.contact_list_builds() >= 2


def test_direct_evaluations_between_steps_force_a_rebuild():
    """rhs() and contact_forces() rebuild the cell structures for the current state; the next
    step rebuilds the list, and the run matches one without the interruption."""
    p = _touching(40, 0.08, 21)
    a = _gpu(p, 3e-4)
    a.step(50, 2e-6)
    a.step(50, 2e-6)
    b = _gpu(p, 3e-4)
    b.step(50, 2e-6)
    n0 = b.contact_list_builds()
    b.rhs(0.0)
    b.contact_forces()
    b.step(50, 2e-6)
    assert b.contact_list_builds() >= n0 + 1
    assert np.abs(a.get_state()[0] - b.get_state()[0]).max() / 0.08 <= 1e-12


def test_skin_must_be_finite_and_non_negative():
    from paper_2605_13766_gb300 import RodError
    s = _gpu(_touching(10, 0.05, 2), 0.0)
    for bad in (-1e-3, float("nan"), float("inf")):
        with pytest.raises(RodError):
            s.contact_skin(bad)
    s.contact_skin(0.0)
    assert s.contact_list_builds() == 0


def test_replayed_graph_launches_rebuild_kernels_only_when_due():
    """Inside a replayed graph the rebuild kernels sit in a conditional node that the device-side
    decision opens only when a rebuild is due: per step the decision, the forces, the step and
    the time advance, plus the eleven rebuild kernels per rebuild.  Eager steps launch all
    fourteen of theirs (decision, eleven rebuild kernels that return at once when no rebuild is due, forces,
    step)."""
    p = _touching(60, 0.1, 14)
    counts = {}
    for graphs in (True, False):
        s = _gpu(p, 2e-4, graphs=graphs)
        s.step(1, 2e-6)                       # grid set-up and the first list build
        b0, l0 = s.contact_list_builds(), s.launch_count
        s.step(65, 2e-6)                      # kinematic half step, 2 graph replays of 32 steps, 1 eager step
        counts[graphs] = (s.contact_list_builds() - b0, s.launch_count - l0)
        s.close()
    (builds_g, n_g), (builds_e, n_e) = counts[True], counts[False]
    assert builds_g == builds_e >= 1
    assert n_e == 1 + 65 * 14
    # kinematic half step, set_time, 64 replayed steps, one eager step with all its kernels
    assert n_g <= 1 + 1 + 64 * 4 + 11 * builds_g + 14
    assert n_g >= 1 + 1 + 64 * 4 + 14



@pytest.mark.parametrize("K", [2, 20, 45])
def test_any_step_count_replays_graphs(K):
    """A call of any length replays graphs for all but its last step: the 32-step graph while
    32 or more steps remain, then the one-step graph; the trajectory is that of eager launches
    bit for bit."""
    p = _touching(60, 0.1, 14)
    counts, states = {}, {}
    for graphs in (True, False):
        s = _gpu(p, 2e-4, graphs=graphs)
        s.step(1, 2e-6)
        b0, l0 = s.contact_list_builds(), s.launch_count
        s.step(K, 2e-6)
        counts[graphs] = (s.contact_list_builds() - b0, s.launch_count - l0)
        states[graphs] = s.get_state()
        s.close()
    for a, b in zip(states[True], states[False]):
        assert np.array_equal(a, b)
    (builds_g, n_g), (builds_e, n_e) = counts[True], counts[False]
    assert builds_g == builds_e
    assert n_e == 1 + K * 14
    # kinematic half step, set_time, K - 1 replayed steps of 4 kernels, the last step eager
    assert 1 + 1 + (K - 1) * 4 + 14 <= n_g <= 1 + 1 + (K - 1) * 4 + 11 * builds_g + 14


def test_replayed_graph_follows_parameter_changes_between_calls():
    """A graph captured for the contact steps is replayed only while nothing baked into it has
    changed: friction set between two step calls, new rest curvatures and element couples, and
    the same state set again give the trajectory of eager launches bit for bit."""
    p = _touching(60, 0.1, 23)
    rng = np.random.default_rng(4)
    kappa = rng.normal(0.0, 0.5, (3, p.n_elems - p.n_rods))
    couple = rng.normal(0.0, 1e-7, (3, p.n_elems))
    out = []
    for graphs in (True, False):
        s = _gpu(p, 2e-4, graphs=graphs)
        s.step(40, 2e-6)
        s.friction(0.4, 1e-3)
        s.step(40, 2e-6)
        s.set_params(kappa, couple)
        s.step(40, 2e-6)
        x, v, Q, w = s.get_state()
        s.set_state(x, v, Q, w)
        s.step(40, 2e-6)
        out.append(s.get_state())
        s.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
