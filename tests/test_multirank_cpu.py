"""Host logic of the multi-GPU benchmark path on CPU: world_size 2 over gloo.

Cells are independent shards (no data-path collective); the only
cross-rank operations are the timing barrier and the max-over-ranks of the
step time.  Each rank also draws its own seeded shard."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = bench.dist_env()
    bench.barrier(w)
    t = bench.allreduce_max(10.0 + rank, w)
    cells, off, bdt, cd, desc = bench.make_workload("uniform4096", r)
    q.put((rank, t, float(cells["n_H"][0]), desc["cells"]))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_shards():
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
    assert res[0][1] == res[1][1] == 11.0          # max over ranks
    assert res[0][2] != res[1][2]                  # independent seeded shards
    assert res[0][3] == res[1][3] == 4096          # same per-rank work (weak scaling)
