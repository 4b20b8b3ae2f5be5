"""Pins of the oracle's derivatives.

* The dual-number build of the oracle (oracle_ad.cpp) advances the state bit for bit like the
  oracle, is linear in its tangents, gives the closed-form tangent of a rigid translation
  (x_N = x_0 + N dt v for a free rod without loads), and agrees with central differences of
  one oracle step.
* The reverse sweep (discrete adjoint built from exact one-step Jacobians) equals the forward
  accumulation of the same gradient entry by entry, and central differences of the oracle's
  own multi-step loss along random directions.
"""
import numpy as np

import rodgen
from oracle.oracle import Oracle
from oracle.reverse_sweep import forward_gradient, reverse_sweep


def tiny_problem():
    p = rodgen.adjoint_batch(n_rods=2, n=5, kappa_scale=2.0, couple_scale=2e-6, target_scale=0.01, seed=13)
    p = p.replace(clamp_base=np.array([1, 0], dtype=np.int8), nu_damp=0.02, gravity=np.array([0.0, -3.0, 0.0]))
    return rodgen.perturbed(p, seed=13, pos=0.01, vel=0.05, rot=0.03, omega=2.0)


def weights(p, seed=3):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=a.shape) for a in p.state()]


def state_loss(W, state):
    """L = sum of seeded weights times every entry of the final state (sensitive to the
    parameters within a few steps through the angular velocities)."""
    return float(sum((w * a).sum() for w, a in zip(W, state)))


def _loss(p, W, kappa0, couple, n_steps, dt):
    q = p.replace(rest_kappa=kappa0, elem_couple=couple)
    return state_loss(W, Oracle(q).step(*q.state(), dt=dt, n_steps=n_steps))


def test_reverse_sweep_matches_finite_differences_of_the_oracle():
    p = tiny_problem()
    n_steps, dt = 12, 1e-5
    W = weights(p)
    gk, gc, _ = reverse_sweep(p, n_steps, dt, W)
    rng = np.random.default_rng(2)
    ks, cs = np.abs(p.rest_kappa).max(), np.abs(p.elem_couple).max()
    def fd(dk, dc, h):
        return (_loss(p, W, p.rest_kappa + h * dk, p.elem_couple + h * dc, n_steps, dt)
                - _loss(p, W, p.rest_kappa - h * dk, p.elem_couple - h * dc, n_steps, dt)) / (2 * h)

    # random directions in both parameter sets, then in the couples alone (their share of the
    # loss is small, so they get a test of their own); Richardson's extrapolation of central
    # differences at h and 2h removes the O(h^2) truncation
    cases = [(rng.normal(size=p.rest_kappa.shape) * ks, rng.normal(size=p.elem_couple.shape) * cs) for _ in range(3)]
    cases += [(np.zeros_like(p.rest_kappa), rng.normal(size=p.elem_couple.shape) * cs) for _ in range(2)]
    for dk, dc in cases:
        # the loss is linear in the couples to ~1e-9 over h = 0.1 (the couple-only differences
        # agree from h = 0.1 to 10), while at h = 1e-4 their rounding is 2e-5 of the result
        h = 1e-4 if np.any(dk) else 0.1
        ref = (4 * fd(dk, dc, h) - fd(dk, dc, 2 * h)) / 3
        ad = float((gk * dk).sum() + (gc * dc).sum())
        assert abs(ad - ref) <= 1e-6 * abs(ref), (ad, ref)
    assert np.abs(gc).max() > 0 and np.abs(gk).max() > 0


def test_dual_step_advances_the_state_like_the_oracle_and_is_linear_in_its_tangents():
    p = tiny_problem()
    o = Oracle(p)
    rng = np.random.default_rng(7)
    tg = [rng.normal(size=a.shape) for a in p.state()]
    dk = rng.normal(size=p.rest_kappa.shape)
    dc = rng.normal(size=p.elem_couple.shape) * 1e-6
    ref = o.step(*p.state(), dt=1e-5, n_steps=7, t=0.2)
    st, t1 = o.step_jvp(p.state(), tg, 1e-5, 7, t=0.2, d_rest_kappa=dk, d_elem_couple=dc)
    for a, b in zip(st, ref):
        assert np.array_equal(a, b)
    # doubling every tangent doubles the result exactly (a power of two scales without rounding)
    _, t2 = o.step_jvp(p.state(), [2 * a for a in tg], 1e-5, 7, t=0.2, d_rest_kappa=2 * dk, d_elem_couple=2 * dc)
    for a, b in zip(t1, t2):
        assert np.array_equal(2 * a, b)
    # sum of two tangents: the sum of the two results to rounding
    tg2 = [rng.normal(size=a.shape) for a in p.state()]
    _, ta = o.step_jvp(p.state(), tg, 1e-5, 7, t=0.2)
    _, tb = o.step_jvp(p.state(), tg2, 1e-5, 7, t=0.2)
    _, tab = o.step_jvp(p.state(), [a + b for a, b in zip(tg, tg2)], 1e-5, 7, t=0.2)
    for a, b, c in zip(ta, tb, tab):
        assert np.abs(a + b - c).max() <= 1e-10 * max(np.abs(c).max(), 1e-300)


def test_dual_tangent_of_a_rigid_translation_is_exact():
    # a free, bent rod without loads: a uniform velocity tangent moves it rigidly, so the
    # position tangent after N steps is N dt dv and the velocity tangent stays dv
    p = rodgen.perturbed(rodgen.cantilever(n=12), seed=9, pos=0.01, vel=0.0, rot=0.02, omega=0.0)
    p = p.replace(clamp_base=None, tip_force=None, nu_damp=0.0, stokes_gamma=0.0, gravity=np.zeros(3))
    o = Oracle(p)
    dv = np.array([0.3, -0.2, 0.5])
    tg = [np.zeros_like(a) for a in p.state()]
    tg[1][:] = dv[:, None]
    n, dt = 9, 1e-5
    _, out = o.step_jvp(p.state(), tg, dt, n)
    assert np.abs(out[0] - n * dt * dv[:, None]).max() <= 1e-12 * n * dt
    assert np.abs(out[1] - dv[:, None]).max() <= 1e-10
    assert np.abs(out[2]).max() <= 1e-10 and np.abs(out[3]).max() <= 1e-6


def test_dual_step_matches_central_differences_of_one_oracle_step():
    p = tiny_problem()
    o = Oracle(p)
    rng = np.random.default_rng(11)
    base = p.state()
    # directions on the state (directors turned along SO(3) tangents) and the parameters
    u = [rng.normal(size=a.shape) * s for a, s in zip(base, (1e-3, 1e-2, 0.0, 1.0))]
    Qb = base[2]
    for e in range(p.n_elems):
        M = Qb[:, e].reshape(3, 3)
        a = rng.normal(size=3)
        K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
        u[2][:, e] = (K @ M).reshape(9)
    dk = rng.normal(size=p.rest_kappa.shape)
    dc = rng.normal(size=p.elem_couple.shape) * np.abs(p.elem_couple).max()
    _, jvp = o.step_jvp(base, u, 1e-5, 1, d_rest_kappa=dk, d_elem_couple=dc)

    def run(h):
        q = p.replace(rest_kappa=p.rest_kappa + h * dk, elem_couple=p.elem_couple + h * dc)
        return Oracle(q).step(*[b + h * du for b, du in zip(base, u)], dt=1e-5, n_steps=1)

    for h in (1e-6,):
        plus, minus = run(h), run(-h)
        for a_idx in (0, 1, 3):
            fd = (plus[a_idx] - minus[a_idx]) / (2 * h)
            assert np.abs(jvp[a_idx] - fd).max() <= 1e-6 * np.abs(fd).max(), a_idx


def test_reverse_sweep_equals_forward_accumulation_entry_by_entry():
    p = tiny_problem()
    n_steps, dt = 12, 1e-5
    W = weights(p)
    gk, gc, _ = reverse_sweep(p, n_steps, dt, W)
    fk, fc = forward_gradient(p, n_steps, dt, W)
    assert np.abs(gk - fk).max() <= 1e-11 * np.abs(fk).max()
    assert np.abs(gc - fc).max() <= 1e-11 * np.abs(fc).max()
