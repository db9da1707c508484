"""Multi-process (world size 2, gloo, CPU) check of the replica aggregation used by
bench.py under torchrun: slowest rank's time, sum of all ranks' frames."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, frames = bench.aggregate_ranks(100.0 + 50.0 * rank, 200 * (rank + 1), world, "cpu")
    q.put((rank, ms, frames))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 150.0, 600), (1, 150.0, 600)]


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(12.5, 40, 1) == (12.5, 40)
