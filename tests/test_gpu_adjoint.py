"""Hand-written adjoint of the rod step (torch.autograd.Function over rod_system_backward).

Gradients of the tip-target loss L = sum_r |x_tip,r(T) - target_r|^2 with respect to the rest
curvature kappa0 and the element couples C are checked against central finite differences
(h = 1e-6) along 8 seeded random directions:
  * small ensemble: differences of the CPU oracle's own forward runs (independent code);
  * the full 1024 x 64 x 2000-step workload: differences of the GPU forward (the forward is
    pinned to the oracle by the parity tests); checkpoint every 100 steps; the 1e-6 check is
    against Richardson-extrapolated differences (h = 1e-3, 2e-3), since at h = 1e-6 the
    differences carry FP64 rounding noise of up to 3e-5 of a directional derivative.
The adjoint of the initial state after one step is also checked entry by entry against
finite differences of the oracle, and the gradients against the oracle's exact derivatives:
its dual-number build (directional derivatives along random directions, on the small ensemble
and on sampled rods of the full workload) and its reverse sweep built from exact one-step
Jacobians (every gradient entry).
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


def _small_problem():
    p = rodgen.adjoint_batch(n_rods=4, n=16, kappa_scale=2.0, couple_scale=2e-6, target_scale=0.01, seed=5)
    clamp = np.array([1, 1, 1, 0], dtype=np.int8)
    rng = np.random.default_rng(5)
    v = p.v.copy()
    off = p.node_offsets()
    v[:, off[3]:off[4]] = rng.normal(0, 0.05, (3, 1))
    return p.replace(clamp_base=clamp, v=v, nu_damp=0.02, gravity=np.array([0.0, -3.0, 0.0]))


def _loss_oracle(p, kappa0, couple, n_steps, dt):
    q = p.replace(rest_kappa=kappa0, elem_couple=couple)
    x = Oracle(q).step(*q.state(), dt=dt, n_steps=n_steps)[0]
    tips = x[:, p.node_offsets()[1:] - 1]
    return float(((tips - p.extra["targets"]) ** 2).sum())


def _jvp_loss_oracle(p, dk, dc, n_steps, dt, targets=None):
    """Exact directional derivative of the tip loss along (dk, dc) by the oracle's dual-number
    build: one forward run of the tangents, no difference quotient."""
    o = Oracle(p)
    zero = [np.zeros_like(a) for a in p.state()]
    st, tg = o.step_jvp(p.state(), zero, dt, n_steps, d_rest_kappa=dk, d_elem_couple=dc)
    tips = p.node_offsets()[1:] - 1
    tgt = p.extra["targets"] if targets is None else targets
    return float((2.0 * (st[0][:, tips] - tgt) * tg[0][:, tips]).sum())


def _grads_gpu(p, n_steps, dt, every):
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300.autograd import rollout, tip_indices
    s = RodSystem(p)
    k0 = torch.tensor(p.rest_kappa, device="cuda", requires_grad=True)
    c0 = torch.tensor(p.elem_couple, device="cuda", requires_grad=True)
    state0 = [torch.tensor(a, device="cuda") for a in p.state()]
    x, v, Q, w = rollout(s, k0, c0, state0, n_steps, dt, every)
    tips = x[:, tip_indices(p.node_offsets())]
    L = ((tips - torch.tensor(p.extra["targets"], device="cuda")) ** 2).sum()
    L.backward()
    return float(L.item()), k0.grad.cpu().numpy(), c0.grad.cpu().numpy(), s


def _directions(p, n, seed):
    rng = np.random.default_rng(seed)
    ks = np.abs(p.rest_kappa).max()
    cs = np.abs(p.elem_couple).max()
    return [(rng.normal(size=p.rest_kappa.shape) * ks, rng.normal(size=p.elem_couple.shape) * cs) for _ in range(n)]


def test_adjoint_matches_oracle_finite_differences_small():
    p = _small_problem()
    n_steps, dt, every = 200, 1e-5, 50
    L, gk, gc, _ = _grads_gpu(p, n_steps, dt, every)
    L_ref = _loss_oracle(p, p.rest_kappa, p.elem_couple, n_steps, dt)
    assert abs(L - L_ref) <= 1e-10 * abs(L_ref)
    report = []
    for dk, dc in _directions(p, 8, seed=1):
        fd = {}
        for h in (1e-6, 1e-5):
            fd[h] = (_loss_oracle(p, p.rest_kappa + h * dk, p.elem_couple + h * dc, n_steps, dt)
                     - _loss_oracle(p, p.rest_kappa - h * dk, p.elem_couple - h * dc, n_steps, dt)) / (2 * h)
        ad = float((gk * dk).sum() + (gc * dc).sum())
        report.append((ad, fd[1e-6], fd[1e-5]))
        assert abs(ad - fd[1e-6]) <= 1e-6 * abs(fd[1e-6]), (ad, fd)
    _record("adjoint_small_oracle_fd", report)


def test_adjoint_matches_the_oracle_dual_derivative_small():
    """The same gradients against the exact directional derivatives of the oracle (its source
    over dual numbers), where finite differences allowed only 1e-6."""
    p = _small_problem()
    n_steps, dt, every = 200, 1e-5, 50
    _, gk, gc, _ = _grads_gpu(p, n_steps, dt, every)
    for dk, dc in _directions(p, 8, seed=1):
        ref = _jvp_loss_oracle(p, dk, dc, n_steps, dt)
        ad = float((gk * dk).sum() + (gc * dc).sum())
        assert abs(ad - ref) <= 1e-9 * abs(ref), (ad, ref)


def test_adjoint_full_workload_matches_the_oracle_dual_derivative_on_sampled_rods():
    """The full 1024 x 64 x 2000-step gradient, restricted to 16 sampled rods, against the exact
    directional derivatives of the oracle run on those rods alone (the rods are clamped and
    touch nothing, so the loss is a sum of independent per-rod terms)."""
    p = rodgen.adjoint_batch()
    n_steps, dt, every = 2000, 1e-5, 100
    _, gk, gc, _ = _grads_gpu(p, n_steps, dt, every)
    eo, R = p.elem_offsets(), p.n_rods
    for r0 in (0, 8, 517, 1016):
        r1 = r0 + 4
        q = p.take_rods(r0, r1)
        e0, e1 = int(eo[r0]), int(eo[r1])
        v0, v1 = e0 - r0, e1 - r1
        rng = np.random.default_rng(r0)
        dk = rng.normal(size=(3, v1 - v0)) * np.abs(q.rest_kappa).max()
        dc = rng.normal(size=(3, e1 - e0)) * np.abs(q.elem_couple).max()
        ref = _jvp_loss_oracle(q, dk, dc, n_steps, dt, targets=p.extra["targets"][:, r0:r1])
        ad = float((gk[:, v0:v1] * dk).sum() + (gc[:, e0:e1] * dc).sum())
        assert abs(ad - ref) <= 1e-8 * abs(ref), (r0, ad, ref)


def test_adjoint_with_magnetic_and_muscle_couples_matches_oracle_finite_differences():
    """The same check with a rotating-field magnetic couple (which depends on the directors)
    and travelling-wave muscle couples on every rod."""
    p = _small_problem()
    rng = np.random.default_rng(8)
    mag = np.zeros((3, p.n_elems))
    mag[2] = rng.uniform(0.5, 1.5, p.n_elems)
    mag[0] = rng.normal(0, 0.3, p.n_elems)
    p = p.replace(magnetization=mag, field_b0=np.array([0.0, 0.0, 1e-3]), field_bc=np.array([4e-3, 0.0, 0.0]),
                  field_bs=np.array([0.0, 4e-3, 0.0]), field_omega=2 * np.pi * 20.0,
                  muscle_amp=np.full(p.n_rods, 2e-6), muscle_period=np.full(p.n_rods, 0.01),
                  muscle_wavelength=np.full(p.n_rods, 0.05), muscle_phase=np.linspace(0, 3, p.n_rods))
    n_steps, dt, every = 200, 1e-5, 50
    L, gk, gc, _ = _grads_gpu(p, n_steps, dt, every)
    L_ref = _loss_oracle(p, p.rest_kappa, p.elem_couple, n_steps, dt)
    assert abs(L - L_ref) <= 1e-10 * abs(L_ref)
    def cd(dk, dc, h):
        return (_loss_oracle(p, p.rest_kappa + h * dk, p.elem_couple + h * dc, n_steps, dt)
                - _loss_oracle(p, p.rest_kappa - h * dk, p.elem_couple - h * dc, n_steps, dt)) / (2 * h)

    for dk, dc in _directions(p, 6, seed=4):
        # Richardson's extrapolation of central differences at h = 1e-4 and 2e-4: at h = 1e-6
        # the rounding of the loss reaches 1e-6 of the smaller directional derivatives here
        fd = (4 * cd(dk, dc, 1e-4) - cd(dk, dc, 2e-4)) / 3
        ad = float((gk * dk).sum() + (gc * dc).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_adjoint_with_a_wall_matches_oracle_finite_differences():
    """Two of the rods press into a side wall during the whole run (normal spring-dashpot;
    friction is checked by the one-step state adjoint, where no slip threshold is crossed)."""
    p = _small_problem().replace(wall_point=np.array([[0.003, 0.0, 0.0]]), wall_normal=np.array([[-1.0, 0.0, 0.0]]),
                                 wall_k=50.0, wall_c=0.01)
    n_steps, dt, every = 200, 1e-5, 50
    L, gk, gc, _ = _grads_gpu(p, n_steps, dt, every)
    L_ref = _loss_oracle(p, p.rest_kappa, p.elem_couple, n_steps, dt)
    assert abs(L - L_ref) <= 1e-10 * abs(L_ref)

    def cd(dk, dc, h):
        return (_loss_oracle(p, p.rest_kappa + h * dk, p.elem_couple + h * dc, n_steps, dt)
                - _loss_oracle(p, p.rest_kappa - h * dk, p.elem_couple - h * dc, n_steps, dt)) / (2 * h)

    for dk, dc in _directions(p, 4, seed=6):
        fd = (4 * cd(dk, dc, 1e-4) - cd(dk, dc, 2e-4)) / 3
        ad = float((gk * dk).sum() + (gc * dc).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_adjoint_full_workload_matches_finite_differences():
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300.autograd import tip_indices
    p = rodgen.adjoint_batch()                       # 1024 rods x 64 elements
    n_steps, dt, every = 2000, 1e-5, 100
    L, gk, gc, s = _grads_gpu(p, n_steps, dt, every)
    tips = tip_indices(p.node_offsets())
    targets = torch.tensor(p.extra["targets"], device="cuda")
    state0 = [torch.tensor(a, device="cuda") for a in p.state()]

    def loss(k, c):
        s.set_params(k, c)
        s.set_state(*state0)
        s.forward_checkpointed(n_steps, dt, every)
        x = s.get_state(device=True)[0]
        return float(((x[:, tips] - targets) ** 2).sum().item())

    # A central difference carries the loss's FP64 rounding noise divided by 2h: here about
    # 6e-15 absolute (a loss of ~0.2 summed over 1024 rods after 2000 steps), i.e. ~3e-9 at
    # h = 1e-6 and up to ~3e-5 of the smaller directional derivatives, so a 1e-6 agreement can
    # only be checked against a difference with less noise: Richardson's extrapolation of the
    # central differences at h = 1e-3 and 2e-3 (noise ~1e-11, truncation O(h^4) on a loss that
    # is smooth at that scale).  The adjoint must agree with it to 1e-6; the h = 1e-6
    # differences are recorded beside it and must agree within their own noise (1e-4).
    k0 = torch.tensor(p.rest_kappa, device="cuda")
    c0 = torch.tensor(p.elem_couple, device="cuda")
    report = []
    for dk, dc in _directions(p, 8, seed=2):
        dkt, dct = torch.tensor(dk, device="cuda"), torch.tensor(dc, device="cuda")
        fd = {}
        for h in (1e-6, 1e-3, 2e-3):
            fd[h] = (loss(k0 + h * dkt, c0 + h * dct) - loss(k0 - h * dkt, c0 - h * dct)) / (2 * h)
        rich = (4.0 * fd[1e-3] - fd[2e-3]) / 3.0
        ad = float((gk * dk).sum() + (gc * dc).sum())
        report.append((ad, fd[1e-6], rich))
        assert abs(ad - rich) <= 1e-6 * abs(rich), (ad, rich, fd)
        assert abs(ad - fd[1e-6]) <= 1e-4 * abs(rich), (ad, rich, fd)
    _record("adjoint_full_fd", report)


def _record(name, rows):
    import json
    import os
    out = os.environ.get("ROD_TEST_RECORD_DIR")   # records are written only when asked for
    if out and os.path.isdir(out):
        with open(os.path.join(out, f"{name}.json"), "w") as f:
            json.dump([{"adjoint": a, "fd_h1e-6": b, "fd_reference": c, "rel_err_h1e-6": abs(a - b) / abs(c),
                        "rel_err_reference": abs(a - c) / abs(c)} for a, b, c in rows], f, indent=1)


@pytest.mark.parametrize("magnetic,wall", [(False, False), (True, False), (False, True)])
def test_state_adjoint_of_one_step_matches_oracle(magnetic, wall):
    """d L / d(initial state) after one step against central differences of the oracle
    (positions, velocities, angular velocities entry by entry; directors along rotations),
    without and with a magnetic couple (which depends on the directors)."""
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300.autograd import rollout, tip_indices
    p = rodgen.perturbed(_small_problem(), seed=9, pos=0.01, vel=0.1, rot=0.05, omega=5.0)
    if magnetic:
        mag = np.zeros((3, p.n_elems))
        mag[2] = 2.0
        mag[1] = 0.5
        p = p.replace(magnetization=mag, field_b0=np.array([3e-2, -2e-2, 1e-2]))
    if wall:
        # a slanted wall that the nodes of the rods at x = 0 press into, sliding along it
        nrm = np.array([-1.0, 0.1, 0.05])
        nrm /= np.linalg.norm(nrm)
        p = p.replace(wall_point=np.array([[0.003, 0.0, 0.0]]), wall_normal=nrm[None, :], wall_k=50.0,
                      wall_c=0.01, wall_mu=0.3, wall_vslip=1e-4, wall_velocity=np.array([[0.0, 0.0, 0.2]]))
    dt = 1e-5
    s = RodSystem(p)
    k0 = torch.tensor(p.rest_kappa, device="cuda", requires_grad=True)
    c0 = torch.tensor(p.elem_couple, device="cuda", requires_grad=True)
    state0 = [torch.tensor(a, device="cuda") for a in p.state()]
    # loss of the whole final state: sum of seeded weights times every state entry
    rng = np.random.default_rng(3)
    W = [rng.normal(size=a.shape) for a in p.state()]
    out = rollout(s, k0, c0, state0, 1, dt, 1)
    L = sum((o * torch.tensor(wt, device="cuda")).sum() for o, wt in zip(out, W))
    L.backward()
    adj = [a.cpu().numpy() for a in s.adjoint_of_state()]
    o = Oracle(p)

    def loss(st):
        fin = o.step(*st, dt=dt, n_steps=1)
        return sum(float((f * wt).sum()) for f, wt in zip(fin, W))

    base = list(p.state())
    # the loss is ~1.4e3, so a central difference carries ~1e-16 * 1.4e3 / (2h) of rounding:
    # 1.5e-5 at h = 1e-8 (the size of the tolerance), 7e-9 at h = 1e-5, where the truncation
    # error of this one-step loss is below 1e-8 (differences at h = 1e-4 and 1e-5 agree to 6e-9)
    h = 1e-5
    checked = 0
    # the clamp holds node 0 and element 0 of a clamped rod at their given values: skip them
    free_nodes = np.ones(p.n_nodes, dtype=bool)
    free_elems = np.ones(p.n_elems, dtype=bool)
    for r in np.flatnonzero(p.clamp_base):
        free_nodes[p.node_offsets()[r]] = False
        free_elems[p.elem_offsets()[r]] = False
    touching = np.ones(p.n_nodes, dtype=bool)
    if wall:
        # the entries of the nodes in contact with the wall (where its force acts)
        pen = p.radius[0] - (p.wall_normal[0][:, None] * (p.x - p.wall_point[0][:, None])).sum(axis=0)
        touching = pen > 0
        assert touching[free_nodes].sum() >= 2
    for a_idx in (0, 1, 3):
        arr = base[a_idx]
        mask = np.broadcast_to(free_nodes & touching if a_idx < 2 else free_elems, arr.shape)
        flat = np.flatnonzero(mask)
        for f in rng.choice(flat, size=min(24, flat.size), replace=False):
            plus = [b.copy() for b in base]
            minus = [b.copy() for b in base]
            plus[a_idx].flat[f] += h
            minus[a_idx].flat[f] -= h
            fd = (loss(plus) - loss(minus)) / (2 * h)
            ad = adj[a_idx].flat[f]
            scale = max(abs(fd), 1e-3 * np.abs(adj[a_idx]).max(), 1e-12)
            assert abs(ad - fd) <= 1e-5 * scale, (a_idx, f, ad, fd)
            checked += 1
    # directors: along tangent directions of SO(3), Q_e <- exp(h [u]x) Q_e (a single entry of Q
    # would leave the rotations, where the two sides' rotation-log formulas are different
    # functions); the adjoint's directional derivative is sum(adj_Q * [u]x Q_e)
    from scipy.spatial.transform import Rotation
    E = p.n_elems
    Qb = base[2]
    for e in rng.choice(np.flatnonzero(free_elems), size=12, replace=False):
        M = Qb[:, e].reshape(3, 3)
        u = rng.normal(size=3)
        K = np.array([[0.0, -u[2], u[1]], [u[2], 0.0, -u[0]], [-u[1], u[0], 0.0]])
        fdv = []
        for sgn in (1.0, -1.0):
            st = [b.copy() for b in base]
            st[2][:, e] = (Rotation.from_rotvec(sgn * h * u).as_matrix() @ M).reshape(9)
            fdv.append(loss(st))
        fd = (fdv[0] - fdv[1]) / (2 * h)
        ad = float((adj[2][:, e].reshape(3, 3) * (K @ M)).sum())
        scale = max(abs(fd), 1e-3 * np.abs(adj[2]).max(), 1e-12)
        assert abs(ad - fd) <= 1e-5 * scale, (e, ad, fd)
        checked += 1
    assert checked > (40 if wall else 60)


def test_adjoint_matches_the_oracle_reverse_sweep():
    """Every entry of the GPU gradients with respect to the rest curvature and the element
    couples, and the adjoint of the free initial positions, velocities and angular velocities,
    against the oracle's reverse sweep (discrete adjoint composed from one-step Jacobians of the
    oracle) on a two-rod problem over 12 steps."""
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300.autograd import rollout
    from oracle.reverse_sweep import reverse_sweep
    from test_oracle_reverse_sweep import tiny_problem, weights
    p = tiny_problem()
    n_steps, dt = 12, 1e-5
    W = weights(p)
    gk_ref, gc_ref, lam_ref = reverse_sweep(p, n_steps, dt, W)
    s = RodSystem(p)
    k0 = torch.tensor(p.rest_kappa, device="cuda", requires_grad=True)
    c0 = torch.tensor(p.elem_couple, device="cuda", requires_grad=True)
    state0 = [torch.tensor(a, device="cuda") for a in p.state()]
    out = rollout(s, k0, c0, state0, n_steps, dt, 4)
    L = sum((o * torch.tensor(wt, device="cuda")).sum() for o, wt in zip(out, W))
    L.backward()
    gk, gc = k0.grad.cpu().numpy(), c0.grad.cpu().numpy()
    # the sweep is exact (dual-number Jacobians), so every entry agrees to 1e-9 of the largest
    assert np.abs(gk - gk_ref).max() <= 1e-9 * np.abs(gk_ref).max(), np.abs(gk - gk_ref).max() / np.abs(gk_ref).max()
    assert np.abs(gc - gc_ref).max() <= 1e-9 * np.abs(gc_ref).max(), np.abs(gc - gc_ref).max() / np.abs(gc_ref).max()
    adj = [a.cpu().numpy() for a in s.adjoint_of_state()]
    free_nodes = np.ones(p.n_nodes, dtype=bool)
    free_elems = np.ones(p.n_elems, dtype=bool)
    for r in np.flatnonzero(p.clamp_base):
        free_nodes[p.node_offsets()[r]] = False
        free_elems[p.elem_offsets()[r]] = False
    for a_idx, mask in ((0, free_nodes), (1, free_nodes), (3, free_elems)):
        got, ref = adj[a_idx][:, mask], lam_ref[a_idx][:, mask]
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (a_idx, np.abs(got - ref).max() / np.abs(ref).max())
