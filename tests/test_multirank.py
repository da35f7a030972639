"""Multi-rank measurement and ensemble sharding, world size 2 over gloo on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2001_11220_gb300.parallel import aggregate, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units, thr = aggregate(10.0 * (rank + 1), 1000.0 * (rank + 1))
        mine = list(shard(513, world, rank))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, ms, units, thr, gathered))
    finally:
        dist.destroy_process_group()


def test_aggregate_and_shard_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, thr, gathered in res:
        assert ms == 20.0                       # max over ranks
        assert units == 3000.0                  # sum over ranks
        assert abs(thr - 3000.0 / 0.02) < 1e-6
        flat = [i for part in gathered for i in part]
        assert flat == list(range(513))         # every instance exactly once, in order


@pytest.mark.parametrize("n,w", [(512, 1), (512, 8), (7, 3), (2, 4)])
def test_shard_partition(n, w):
    parts = [list(shard(n, w, r)) for r in range(w)]
    assert [i for p in parts for i in p] == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_aggregate_single_process():
    ms, units, thr = aggregate(5.0, 100.0)
    assert (ms, units) == (5.0, 100.0) and abs(thr - 2e4) < 1e-9
