"""The replicas path of bench.py on two CPU processes (gloo, world size 2).

Each rank runs an independent replica; the job's time is the slowest rank's
(max over ranks), the job's rate every rank's units over that time, every rank
draws its own workload instance, and under the reference arm only rank 0 works.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = [0.25, 0.75][rank]          # the second replica is the slow one
        job = bench.max_over_ranks(dist, seconds)
        rate = bench.job_rate(world, 1000, job)
        ref = bench.run_reference(None, rank, world) if rank == 1 else "skipped"
        out[rank] = (job, rate, bench.replica_seed(rank), ref)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        job, rate, seed, _ = res[rank]
        assert job == 0.75
        assert rate == pytest.approx(2 * 1000 / 0.75)
        assert seed == rank + 1
    assert res[0][2] != res[1][2]
    assert res[1][3] is None                  # the reference arm: ranks other than 0 do no work
    assert bench_value_without_group() == 0.5


def bench_value_without_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    return bench.max_over_ranks(None, 0.5)
