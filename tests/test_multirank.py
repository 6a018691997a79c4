"""Multi-rank host logic on CPU (gloo, world size 2): the bench's max-over-ranks timing.

The path has no exchange step (replicas only), so the only cross-rank operation
is the reduction of per-rank timings before rank 0 prints the JSON line.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = [10.0 + rank, 5.0 - rank, 7.0 * (rank + 1)]
    out[rank] = bench.max_over_ranks(vals, dist, "cpu")
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == [11.0, 5.0, 14.0]


def test_max_over_ranks_without_process_group():
    import bench

    assert bench.max_over_ranks([1.0, 2.0], None, "cpu") == [1.0, 2.0]
