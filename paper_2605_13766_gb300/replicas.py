"""Multi-GPU plumbing for independent rod ensembles ("replicas only").

Without contact the rods never exchange data, so a multi-GPU run is one ensemble per rank
(weak scaling) or the rods of one ensemble split into contiguous ranges (strong scaling),
with no collective on the data path.  The only communication is host-side bookkeeping: the
slowest rank's time and the total of the processed units.
"""
from __future__ import annotations

import numpy as np


def shard_rods(n_elem, world: int, rank: int):
    """Contiguous rod range [r0, r1) of ``rank`` with about 1/world of the elements each."""
    n_elem = np.asarray(n_elem, dtype=np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    cum = np.concatenate([[0], np.cumsum(n_elem)])
    total = cum[-1]
    bounds = []
    for k in range(world + 1):
        target = total * k / world
        i = int(np.searchsorted(cum, target, side="left"))
        if i > 0 and (i >= len(cum) or abs(cum[i - 1] - target) <= abs(cum[i] - target)):
            i -= 1                                # the rod boundary nearest to the target
        bounds.append(i)
    bounds[0], bounds[-1] = 0, len(n_elem)
    for k in range(1, world + 1):               # keep ranges ordered when rods are few
        bounds[k] = max(bounds[k], bounds[k - 1])
    return bounds[rank], bounds[rank + 1]


def slowest(t_local: float) -> float:
    """Largest value of ``t_local`` over the ranks of the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(t_local)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def total(units_local: float) -> float:
    """Sum of ``units_local`` over the ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units_local)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
