"""The benchmark's multi-rank aggregation on CPU (gloo, world size 2).

With N GPUs every rank solves its own copy of the system (replicas; the
method has no data-path exchange).  The whole-job rate is N x steps over the
slowest rank's time; this checks the max reduction and the rate on two gloo
ranks, with no GPU.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [250.0, 400.0][rank]  # rank 1 is the slower one
        slow = bench.slowest_rank(dist, local, "cpu")
        out[rank] = (slow, bench.whole_job_rate(world, 5, slow))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1]
    slow, rate = out[0]
    assert slow == pytest.approx(400.0)
    assert rate == pytest.approx(2 * 5 / 0.4)
