"""Multi-process path on the CPU (gloo, world size 2).

The library does not shard one problem across GPUs: N GPUs run N independent
replicas and the benchmark reports the whole job's time per solve, the
slowest rank's time divided by every solve of the job.  This checks that
reduction across two gloo ranks.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_step, value = bench.job_ms_per_solve(100.0 + 50.0 * rank, 5, world)
        out[rank] = (ms_step, value)
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_ranks_per_solve():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # slowest rank: 150 ms for 5 solves -> 30 ms per step; 10 solves in the job
    assert res == {0: (30.0, 15.0), 1: (30.0, 15.0)}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_ms_per_solve(120.0, 4, 1) == (30.0, 30.0)
