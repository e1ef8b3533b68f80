"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups (127.0.0.1), no GPU.
Every rank runs its own replica (the path has no exchange step on one GPU), so the multi-rank
logic is the barrier, the maximum over ranks of the per-step time, and the whole-job value;
rank 0 alone prints.  Ranks that differ in speed must report the slowest time everywhere."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 1.5 if rank == 0 else 2.5           # the second rank is the slow one
        slowest = bench.max_over_ranks(ms, world, torch.device("cpu"))
        value = bench.whole_job_gflops(8.0e9, world, slowest)
        results[rank] = (slowest, value)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = dict(results)
    for r in range(world):
        slowest, value = got[r]
        assert slowest == 2.5
        assert value == pytest.approx(world * 8.0e9 / 2.5e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.whole_job_gflops(4.0e9, 1, 2.0) == pytest.approx(2000.0)
