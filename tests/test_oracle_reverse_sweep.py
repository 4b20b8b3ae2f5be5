"""Pin of the oracle's reverse sweep (discrete adjoint built from one-step Jacobians): its
gradient of a tip-target loss with respect to the rest curvature and the element couples
equals central differences of the oracle's own multi-step loss along random directions."""
import numpy as np

import rodgen
from oracle.oracle import Oracle
from oracle.reverse_sweep import reverse_sweep


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
