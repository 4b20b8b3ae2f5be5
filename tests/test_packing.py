"""Host logic of the thread-block packing (rod_plan_packs, no GPU needed).

Checks the plan the step kernels receive: every rod that fits a block in exactly one pack, the
capacities respected, heaviest packs first, never more packs than packing in index order, and,
replaying the pack staging's index offsets (global element = local + elem0 - rel, global node =
local + node0 - rel - r, global Voronoi point = local + elem0 - g - rel + r for the r-th rod g
of a pack whose first element within the pack is rel), every element, node and Voronoi point
of those rods covered exactly once.  The two benchmark ensembles give the grids their profiled
launches had (5475 blocks for the 10^4-rod packing at 256 x 256, 586 for the 64 x 64 carpet at
384 elements per block).
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def plan():
    from paper_2605_13766_gb300 import build
    build.build()
    from paper_2605_13766_gb300.binding import plan_packs
    return plan_packs


def _consecutive_count(n, cap, cap_rods):
    packs, cur_e, cur_r = 0, 0, 0
    for k in n:
        if k > cap:
            if cur_r:
                packs += 1
            cur_e = cur_r = 0
            continue
        if cur_r and (cur_e + k > cap or cur_r + 1 > cap_rods):
            packs += 1
            cur_e = cur_r = 0
        cur_e += k
        cur_r += 1
    return packs + (1 if cur_r else 0)


def _check(plan, n, cap, cap_rods):
    n = np.asarray(n, dtype=np.int64)
    R = n.size
    elem0 = np.concatenate([[0], np.cumsum(n)[:-1]])
    node0 = elem0 + np.arange(R)
    out = plan(n, cap, cap_rods)
    packs, lst = out["packs"], out["list"]
    assert out["n_long"] == int((n > cap).sum())
    seen_rod = np.zeros(R, dtype=int)
    seen_e = np.zeros(int(n.sum()), dtype=int)
    seen_n = np.zeros(int(n.sum()) + R, dtype=int)
    seen_v = np.zeros(int(n.sum()) - R, dtype=int)
    weights = []
    for rod0, nrods, e0, ne, n0, nn, v0, nv, listed, off in packs:
        assert 1 <= nrods <= cap_rods and ne <= cap
        assert nn == ne + nrods and nv == ne - nrods
        if listed:
            entries = lst[off:off + nrods]
            rods, rels = entries[:, 0], entries[:, 1]
            assert ne + nrods <= cap                      # best fit counts nodes
        else:
            rods = rod0 + np.arange(nrods)
            rels = elem0[rods] - e0
        # the rods' first pack-local elements are the running sums of their lengths
        assert np.array_equal(rels, np.concatenate([[0], np.cumsum(n[rods])[:-1]]))
        assert int(n[rods].sum()) == ne
        for r, (g, rel) in enumerate(zip(rods, rels)):
            k = int(n[g])
            seen_rod[g] += 1
            dE, dN, dV = elem0[g] - rel, node0[g] - rel - r, elem0[g] - g - rel + r
            seen_e[np.arange(rel, rel + k) + dE] += 1
            seen_n[np.arange(rel + r, rel + r + k + 1) + dN] += 1
            seen_v[np.arange(rel - r, rel - r + k - 1) + dV] += 1
        weights.append(ne + nn)
    short = n <= cap
    assert np.array_equal(seen_rod, short.astype(int))
    for arr, owner in ((seen_e, np.repeat(np.arange(R), n)), (seen_n, np.repeat(np.arange(R), n + 1)),
                       (seen_v, np.repeat(np.arange(R), n - 1))):
        assert np.array_equal(arr, short[owner].astype(int))
    assert weights == sorted(weights, reverse=True)
    assert len(packs) <= _consecutive_count(n, cap, cap_rods)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("cap,cap_rods", [(128, 16), (256, 16), (384, 64), (768, 8)])
def test_random_ensembles(plan, seed, cap, cap_rods):
    n = np.random.default_rng(seed).integers(1, 300, 400)
    _check(plan, n, cap, cap_rods)


def test_single_element_rods_and_long_rods(plan):
    n = [1, 1, 2, 900, 1, 3, 383, 1, 2000, 64, 1]
    out = _check(plan, n, 384, 64)
    assert out["n_long"] == 2


def test_equal_rods_keep_consecutive_packs(plan):
    out = _check(plan, np.full(4096, 50), 384, 8)
    assert len(out["packs"]) == 586 and out["list"].size == 0      # 7 rods of 50 per block


def test_benchmark_packing_plan(plan):
    """The 10^4-rod packing (n ~ U{16..256}, seed 1234) at 256 elements and 16 rods per block."""
    n = np.random.default_rng(1234).integers(16, 257, 10000)
    assert n.sum() == 1366295
    out = _check(plan, n, 256, 16)
    assert len(out["packs"]) == 5475 < _consecutive_count(n, 256, 16)
    fill = (out["packs"][:, 5].sum()) / (len(out["packs"]) * 256)
    assert fill > 0.98


def test_invalid_arguments(plan):
    from paper_2605_13766_gb300.binding import RodError
    with pytest.raises(RodError):
        plan([3, 0, 2], 256, 16)
    with pytest.raises(RodError):
        plan([3, 2], 0, 16)
