"""The oracle's reverse sweep: gradients of a loss of the final state with respect to the rest
curvature and the element couples by the discrete adjoint of the oracle's own step.

TEST INFRASTRUCTURE ONLY.  For the step s_{k+1} = F(s_k, theta) (one oracle step of dt from
time k dt) the adjoint recursion is

    lambda_N = dL/ds_N,   lambda_k = (dF/ds_k)^T lambda_{k+1},   dL/dtheta = sum_k (dF/dtheta)^T lambda_{k+1},

with every Jacobian of one oracle step built column by column as exact Jacobian-vector
products of the oracle's source evaluated over dual numbers (oracle_ad.cpp): no difference
quotient and no step size anywhere, so the sweep is the adjoint of the oracle's discrete map up
to rounding (plain, slow and only for small systems: one dual step per state and parameter
entry per step).  The director columns are single entries of Q: off the rotations the chain
differentiates the oracle's own extension of the step, and the final contraction with
dF/dtheta (whose director part is tangent, since each step turns the directors) keeps the
parameter gradient independent of it.

``forward_gradient`` gives the same gradient by the other accumulation order: one dual run of
the whole horizon per parameter entry (the directional derivative along that entry), so the two
agree to rounding and pin each other's bookkeeping.
"""
from __future__ import annotations

import numpy as np

from .oracle import Oracle


def _flat(state):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in state])


def _unflat(vec, shapes):
    out, off = [], 0
    for shp in shapes:
        n = int(np.prod(shp))
        out.append(vec[off:off + n].reshape(shp).copy())
        off += n
    return out


def _params(problem):
    p = problem
    kappa0 = np.array(p.rest_kappa if p.rest_kappa is not None else np.zeros((3, p.n_voronoi)), dtype=np.float64)
    couple0 = np.array(p.elem_couple if p.elem_couple is not None else np.zeros((3, p.n_elems)), dtype=np.float64)
    return kappa0, couple0


def reverse_sweep(problem, n_steps: int, dt: float, dL_dfinal, t0: float = 0.0):
    """(grad_rest_kappa (3, V), grad_elem_couple (3, E), lambda_0 as (x, v, Q, w)) for a loss
    whose gradient with respect to the final state is ``dL_dfinal`` (x, v, Q, w arrays)."""
    p = problem
    state0 = p.state()
    shapes = [a.shape for a in state0]
    kappa0, couple0 = _params(p)
    o = Oracle(p.replace(rest_kappa=kappa0, elem_couple=couple0))

    # forward: keep every state
    states = [_flat(state0)]
    st = state0
    for k in range(n_steps):
        st = o.step(*st, dt=dt, n_steps=1, t=t0 + k * dt)
        states.append(_flat(st))

    zero_state = [np.zeros(s) for s in shapes]
    n_s = states[0].size
    n_k, n_c = kappa0.size, couple0.size

    def column(s_k, k, state_dir=None, dk=None, dc=None):
        """One Jacobian column of step k at state s_k: the tangent of F along the given
        direction of the state or the parameters."""
        tg = zero_state if state_dir is None else _unflat(state_dir, shapes)
        _, out = o.step_jvp(_unflat(s_k, shapes), tg, dt, 1, t=t0 + k * dt, d_rest_kappa=dk, d_elem_couple=dc)
        return _flat(out)

    lam = _flat(dL_dfinal)
    g_k = np.zeros(n_k)
    g_c = np.zeros(n_c)
    for k in range(n_steps - 1, -1, -1):
        s_k = states[k]
        for j in range(n_k):                           # (dF/dkappa0)^T lambda_{k+1}
            e = np.zeros(n_k)
            e[j] = 1.0
            g_k[j] += column(s_k, k, dk=e.reshape(kappa0.shape)) @ lam
        for j in range(n_c):                           # (dF/dC)^T lambda_{k+1}
            e = np.zeros(n_c)
            e[j] = 1.0
            g_c[j] += column(s_k, k, dc=e.reshape(couple0.shape)) @ lam
        new = np.zeros(n_s)                            # lambda_k = (dF/ds_k)^T lambda_{k+1}
        for j in range(n_s):
            e = np.zeros(n_s)
            e[j] = 1.0
            new[j] = column(s_k, k, state_dir=e) @ lam
        lam = new
    return g_k.reshape(kappa0.shape), g_c.reshape(couple0.shape), _unflat(lam, shapes)


def forward_gradient(problem, n_steps: int, dt: float, dL_dfinal, t0: float = 0.0):
    """(grad_rest_kappa, grad_elem_couple) of the same loss by forward accumulation: for each
    parameter entry, the tangent of the final state after n_steps dual steps, contracted with
    dL/ds_N."""
    p = problem
    state0 = p.state()
    kappa0, couple0 = _params(p)
    o = Oracle(p.replace(rest_kappa=kappa0, elem_couple=couple0))
    lam = _flat(dL_dfinal)
    zero = [np.zeros_like(a) for a in state0]
    g_k = np.zeros(kappa0.size)
    g_c = np.zeros(couple0.size)
    for j in range(kappa0.size):
        e = np.zeros(kappa0.size)
        e[j] = 1.0
        _, tg = o.step_jvp(state0, zero, dt, n_steps, t=t0, d_rest_kappa=e.reshape(kappa0.shape))
        g_k[j] = _flat(tg) @ lam
    for j in range(couple0.size):
        e = np.zeros(couple0.size)
        e[j] = 1.0
        _, tg = o.step_jvp(state0, zero, dt, n_steps, t=t0, d_elem_couple=e.reshape(couple0.shape))
        g_c[j] = _flat(tg) @ lam
    return g_k.reshape(kappa0.shape), g_c.reshape(couple0.shape)
