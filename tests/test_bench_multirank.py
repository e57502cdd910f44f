"""World-size-2 check (gloo, CPU) of bench.py's multi-rank timing: every rank
sees the slowest rank's time, and the job throughput counts all ranks' units
over that time (replicas, weak scaling)."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1)
    dist.barrier()
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.job_throughput(1000, 5, world, m)
    dist.barrier()
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == out[1][1] == pytest.approx(1000 * 5 * 2 / 0.020)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(10, 2, 1, 1.0) == pytest.approx(20000.0)
