"""torch.autograd.Function over the hand-written adjoint of the rod step.

``rollout(system, rest_kappa, elem_couple, state0, n_steps, dt, every)`` returns the final
state (x, v, Q, w) as CUDA tensors; gradients of any torch loss of it flow back to the rest
curvature (3, V) and the element couples (3, E) through ``rod_system_backward`` (checkpoint
every ``every`` steps, recompute, reverse sweep in CUDA).  Only argument marshalling happens
here.
"""
from __future__ import annotations

import torch


class RodRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rest_kappa, elem_couple, system, state0, n_steps, dt, every):
        system.set_params(rest_kappa, elem_couple)
        system.set_state(*state0)
        system.forward_checkpointed(n_steps, dt, every)
        x, v, Q, w = system.get_state(device=True)
        ctx.system = system
        return x, v, Q, w

    @staticmethod
    def backward(ctx, gx, gv, gQ, gw):
        s = ctx.system
        z = lambda g, shape: torch.zeros(shape, dtype=torch.float64, device="cuda") if g is None else g
        gx = z(gx, (3, s.n_nodes))
        gv = z(gv, (3, s.n_nodes))
        gQ = z(gQ, (9, s.n_elems))
        gw = z(gw, (3, s.n_elems))
        gk, gc = s.backward(gx, gv, gQ, gw)
        return gk, gc, None, None, None, None, None


def rollout(system, rest_kappa, elem_couple, state0, n_steps: int, dt: float, every: int = 100):
    return RodRollout.apply(rest_kappa, elem_couple, system, state0, int(n_steps), float(dt), int(every))


def tip_indices(node_offsets) -> torch.Tensor:
    """Index of every rod's last node in the packed node arrays."""
    import numpy as np
    return torch.as_tensor(np.asarray(node_offsets)[1:] - 1, dtype=torch.long, device="cuda")
