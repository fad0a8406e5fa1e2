"""The bench's multi-GPU arithmetic (replicas: max time over ranks, units
summed over ranks) on two CPU ranks over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, rate = bench.job_rate(100.0 + 50.0 * rank, 1000.0, torch.device("cpu"))
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == pytest.approx(150.0)  # the slowest rank
        assert rate == pytest.approx(world * 1000.0 / 0.150)


def test_job_rate_single_process():
    import bench

    ms, rate = bench.job_rate(200.0, 1000.0, torch.device("cpu"))
    assert ms == 200.0 and rate == pytest.approx(5000.0)
