"""The multi-GPU path of bench.py runs independent replicas, one per rank
(the single-system evaluation does not shard): each rank times its own steps,
the job's time is the slowest rank's (all-reduce MAX) and the throughput is
world x units per rank / that time.  These two-rank tests run that host logic
over the gloo backend on CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.reduce_max(times[rank], dist, torch.device("cpu"))
        out[rank] = (slowest, bench.aggregate_rate(world, 100, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    times = [0.25, 0.40]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
    for r in range(world):
        slowest, rate = out[r]
        assert slowest == pytest.approx(0.40)
        assert rate == pytest.approx(2 * 100 / 0.40)


def test_single_process_needs_no_collective():
    assert bench.reduce_max(1.5, None, None) == 1.5
    assert bench.aggregate_rate(1, 50, 0.5) == pytest.approx(100.0)
