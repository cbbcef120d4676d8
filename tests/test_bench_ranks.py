"""Multi-rank path of bench.py on CPU (gloo, world size 2): the method runs
as independent replicas, one per GPU, so the only exchange is the timing
reduction -- the job is as slow as its slowest rank and its throughput is
the sum over the replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)           # rank 1 is the slow one
    tot = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (tot, bench.job_value(tot, world, 8, 10))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        tot, value = res[r]
        assert tot == 200.0
        assert abs(value - world * 8 * 10 / 0.2) < 1e-9


def test_single_rank_value():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert abs(bench.job_value(500.0, 1, 8, 10) - 160.0) < 1e-12
