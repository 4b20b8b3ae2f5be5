"""Multi-rank host logic on CPU (gloo, world size 2): rod sharding and the slowest-rank /
total-units aggregation the benchmark uses for N > 1 GPUs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_elem, out):
    import torch.distributed as dist
    from paper_2605_13766_gb300.replicas import shard_rods, slowest, total
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r0, r1 = shard_rods(n_elem, world, rank)
    units = float(np.sum(n_elem[r0:r1]))
    t = 1.0 + rank          # rank 1 is the slow one
    out.put((rank, r0, r1, slowest(t), total(units)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    rng = np.random.default_rng(0)
    n_elem = rng.integers(16, 257, 1000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_elem, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a0, a1, ta, ua), (_, b0, b1, tb, ub) = res
    assert a0 == 0 and a1 == b0 and b1 == len(n_elem)          # contiguous, disjoint, complete
    ea, eb = n_elem[a0:a1].sum(), n_elem[b0:b1].sum()
    assert abs(ea - eb) <= n_elem.max()                        # balanced to one rod
    assert ta == tb == 2.0                                     # slowest rank's time on both
    assert ua == ub == float(n_elem.sum())                     # all units counted once


def test_shard_rods_edge_cases():
    from paper_2605_13766_gb300.replicas import shard_rods
    n = np.array([5, 1, 1, 1])
    got = [shard_rods(n, 3, r) for r in range(3)]
    assert got[0][0] == 0 and got[-1][1] == 4
    assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
    assert shard_rods(n, 1, 0) == (0, 4)
    with pytest.raises(ValueError):
        shard_rods(n, 2, 2)
