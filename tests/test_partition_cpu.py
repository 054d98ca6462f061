"""The multi-device partition of one workload (host only, no GPU):
sfchem_partition cuts a block list into contiguous ranges balanced by each
block's cost (the previous call's substeps), and the ranks of a gloo group
that gather their costs agree on one cut."""
import itertools
import os
import socket

import numpy as np
import pytest

import paper_2604_21438_gb300 as sf


def _brute_bottleneck(cost, parts):
    """Smallest achievable largest-part cost over all contiguous cuts."""
    n = len(cost)
    best = np.inf
    for cuts in itertools.combinations_with_replacement(range(n + 1), parts - 1):
        edges = (0,) + cuts + (n,)
        worst = max(cost[a:b].sum() for a, b in zip(edges, edges[1:]))
        best = min(best, worst)
    return best


def _check_cut(cut, nb, parts):
    assert len(cut) == parts + 1 and cut[0] == 0 and cut[-1] == nb
    assert np.all(np.diff(cut) >= 0)


def test_partition_is_optimal_on_small_cases():
    rng = np.random.default_rng(5)
    for trial in range(200):
        nb = int(rng.integers(1, 9))
        parts = int(rng.integers(1, 5))
        cost = rng.choice([1.0, 2.0, 3.0, 7.0, 40.0], nb) * rng.integers(1, 4, nb)
        off = np.concatenate([[0], np.cumsum(rng.integers(1, 10, nb))]).astype(np.int64)
        cut = sf.partition(off, parts, cost)
        _check_cut(cut, nb, parts)
        got = max(cost[a:b].sum() for a, b in zip(cut[:-1], cut[1:]))
        assert got <= _brute_bottleneck(cost, parts) * (1 + 1e-9), (trial, cost, parts, cut)


def test_partition_balance_bound_and_cell_weights():
    rng = np.random.default_rng(6)
    nb, parts = 3000, 8
    cells = rng.integers(64, 4097, nb)
    off = np.concatenate([[0], np.cumsum(cells)]).astype(np.int64)
    cost = rng.lognormal(5.0, 1.5, nb)
    cut = sf.partition(off, parts, cost)
    _check_cut(cut, nb, parts)
    load = np.array([cost[a:b].sum() for a, b in zip(cut[:-1], cut[1:])])
    assert load.max() <= cost.sum() / parts + cost.max()
    assert load.min() > 0.5 * cost.sum() / parts
    # no costs: balanced by cells
    cut = sf.partition(off, parts)
    lc = np.array([cells[a:b].sum() for a, b in zip(cut[:-1], cut[1:])])
    assert lc.max() <= cells.sum() / parts + cells.max()
    # zero-cost blocks weigh their cells; more parts than blocks leave parts empty
    cut = sf.partition(off[:4], 6, np.zeros(3))
    _check_cut(cut, 3, 6)
    assert (np.diff(cut) > 0).sum() == 3


def test_partition_rejects_bad_arguments():
    off = np.array([0, 4, 8], np.int64)
    with pytest.raises(sf.SfchemError):
        sf.partition(off, 0)
    with pytest.raises(sf.SfchemError):
        sf.partition(np.array([1, 4, 8], np.int64), 2)
    with pytest.raises(sf.SfchemError):
        sf.partition(np.array([0, 4, 2], np.int64), 2)
    with pytest.raises(sf.SfchemError):
        sf.partition(off, 2, np.array([1.0, np.nan]))
    with pytest.raises(sf.SfchemError):
        sf.partition(off, 2, np.array([1.0, -1.0]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # one workload of 40 blocks; each rank first holds a count-balanced range
    # and measured costs for it (here: seeded per-rank numbers)
    nb = 40
    off = np.arange(nb + 1, dtype=np.int64) * 512
    first = sf.partition(off, world)
    lo, hi = int(first[rank]), int(first[rank + 1])
    mine = np.random.default_rng(100 + rank).lognormal(4.0, 1.0, hi - lo)
    cost = bench.gather_block_costs(mine, lo, nb, world)
    cut = sf.partition(off, world, cost)
    q.put((rank, cut.tolist(), cost.tolist()))
    dist.destroy_process_group()


def test_two_ranks_agree_on_a_cost_balanced_cut():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, cut0, cost0), (r1, cut1, cost1) = res
    assert cut0 == cut1 and cost0 == cost1           # one cut, from the same gathered costs
    cost = np.array(cost0)
    # both ranks' measured costs landed in their own range
    assert np.allclose(cost[:20], np.random.default_rng(100).lognormal(4.0, 1.0, 20))
    assert np.allclose(cost[20:], np.random.default_rng(101).lognormal(4.0, 1.0, 20))
    load = [cost[a:b].sum() for a, b in zip(cut0[:-1], cut0[1:])]
    assert max(load) <= cost.sum() / 2 + cost.max()


def test_shard_slabs_covers_each_range_once():
    """The benchmark's multi-device workload is made of equal slabs; a rank's
    contiguous block range maps to pieces of at most a few slabs, in order,
    and the ranks' pieces tile the whole block list exactly once."""
    import bench
    slab_blocks, world = 16, 4
    rng = np.random.default_rng(9)
    off = np.arange(world * slab_blocks + 1, dtype=np.int64) * 64
    cost = rng.lognormal(3.0, 1.0, world * slab_blocks)
    cut = sf.partition(off, world, cost)
    seen = []
    for r in range(world):
        pieces = bench.shard_slabs(cut, r, slab_blocks)
        for s, b0, b1 in pieces:
            assert 0 <= b0 < b1 <= slab_blocks
            seen.extend(range(s * slab_blocks + b0, s * slab_blocks + b1))
        assert sum(b1 - b0 for _, b0, b1 in pieces) == cut[r + 1] - cut[r]
    assert seen == list(range(world * slab_blocks))
