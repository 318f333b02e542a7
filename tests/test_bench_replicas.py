"""bench.py's multi-GPU bookkeeping (replicas only: one independent system per rank, no data-path
collective): timing is the maximum over ranks and the job's rate counts every rank's steps.  Run as two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # the slower rank decides the job's time
        mx = bench.replica_max(dist, ms)
        out[rank] = (mx, bench.job_throughput(world, 1000, mx), bench.make_system_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 1000 / 0.150)
    assert res[0][2] != res[1][2]  # every rank runs its own replica


def test_single_process_needs_no_group():
    assert bench.replica_max(None, 12.5) == 12.5
    assert bench.job_throughput(1, 300, 100.0) == pytest.approx(3000.0)
