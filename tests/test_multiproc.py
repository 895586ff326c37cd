"""The N > 1 path of bench.py on CPU: two gloo ranks aggregate their timings
the way the GPU bench does (max of elapsed time, sum of processed units).
The transform has no exchange step, so this is the only collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.dist_env()
        assert (w, r, lr) == (world, rank, rank)
        elapsed = 10.0 + 5.0 * rank
        units = 100.0 * (rank + 1)
        bench.barrier(world)
        ms, tot = bench.aggregate(elapsed, units, world, torch.device("cpu"))
        q.put((rank, ms, tot))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for _, ms, tot in res:
        assert ms == 15.0      # slowest rank
        assert tot == 300.0    # all ranks' units


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(7.0, 42.0, 1) == (7.0, 42.0)
