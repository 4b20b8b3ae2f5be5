"""The oracle's reverse sweep: gradients of a loss of the final state with respect to the rest
curvature and the element couples by the discrete adjoint of the oracle's own step.

TEST INFRASTRUCTURE ONLY.  For the step s_{k+1} = F(s_k, theta) (one oracle step of dt from
time k dt) the adjoint recursion is

    lambda_N = dL/ds_N,   lambda_k = (dF/ds_k)^T lambda_{k+1},   dL/dtheta = sum_k (dF/dtheta)^T lambda_{k+1},

with every Jacobian of one oracle step built column by column by central differences (so the
sweep is plain, slow and only for small systems: 2 (n_state + n_theta) oracle steps per step).
The director columns perturb single entries of Q: off the rotations the chain uses the
oracle's own extension of the step, and the final contraction with dF/dtheta (whose director
part is tangent, since each step turns the directors) keeps the gradient independent of it.
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


def reverse_sweep(problem, n_steps: int, dt: float, dL_dfinal, h: float = 1e-6, t0: float = 0.0,
                  h_couple: float = 1e-2):
    """(grad_rest_kappa (3, V), grad_elem_couple (3, E), lambda_0 as (x, v, Q, w)) for a loss
    whose gradient with respect to the final state is ``dL_dfinal`` (x, v, Q, w arrays)."""
    p = problem
    state0 = p.state()
    shapes = [a.shape for a in state0]
    kappa0 = np.array(p.rest_kappa if p.rest_kappa is not None else np.zeros((3, p.n_voronoi)), dtype=np.float64)
    couple0 = np.array(p.elem_couple if p.elem_couple is not None else np.zeros((3, p.n_elems)), dtype=np.float64)
    o = Oracle(p.replace(rest_kappa=kappa0, elem_couple=couple0))

    # forward: keep every state
    states = [_flat(state0)]
    st = state0
    for k in range(n_steps):
        st = o.step(*st, dt=dt, n_steps=1, t=t0 + k * dt)
        states.append(_flat(st))

    def step_flat(vec, k, oracle):
        return _flat(oracle.step(*_unflat(vec, shapes), dt=dt, n_steps=1, t=t0 + k * dt))

    n_s = states[0].size
    n_k, n_c = kappa0.size, couple0.size
    lam = _flat(dL_dfinal)
    g_k = np.zeros(n_k)
    g_c = np.zeros(n_c)
    for k in range(n_steps - 1, -1, -1):
        s_k = states[k]
        # parameter part: (dF/dtheta)^T lambda_{k+1}, columns by central differences
        for j in range(n_k):
            dk = np.zeros(n_k)
            dk[j] = h * max(1.0, abs(kappa0.flat[j]))
            op = Oracle(p.replace(rest_kappa=kappa0 + dk.reshape(kappa0.shape), elem_couple=couple0))
            om = Oracle(p.replace(rest_kappa=kappa0 - dk.reshape(kappa0.shape), elem_couple=couple0))
            col = (step_flat(s_k, k, op) - step_flat(s_k, k, om)) / (2 * dk[j])
            g_k[j] += col @ lam
        # a couple enters the step linearly up to the director turn it causes, so its columns
        # take a large step (h_couple x the largest couple): less rounding, same truncation
        cs = max(np.abs(couple0).max(), 1e-9)
        for j in range(n_c):
            dc = np.zeros(n_c)
            dc[j] = h_couple * cs
            op = Oracle(p.replace(rest_kappa=kappa0, elem_couple=couple0 + dc.reshape(couple0.shape)))
            om = Oracle(p.replace(rest_kappa=kappa0, elem_couple=couple0 - dc.reshape(couple0.shape)))
            col = (step_flat(s_k, k, op) - step_flat(s_k, k, om)) / (2 * dc[j])
            g_c[j] += col @ lam
        # state part: lambda_k = (dF/ds_k)^T lambda_{k+1}
        new = np.zeros(n_s)
        for j in range(n_s):
            e = h * max(1.0, abs(s_k[j]))
            sp = s_k.copy()
            sm = s_k.copy()
            sp[j] += e
            sm[j] -= e
            col = (step_flat(sp, k, o) - step_flat(sm, k, o)) / (2 * e)
            new[j] = col @ lam
        lam = new
    return g_k.reshape(kappa0.shape), g_c.reshape(couple0.shape), _unflat(lam, shapes)
