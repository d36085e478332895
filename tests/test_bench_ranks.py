"""The benchmark's multi-rank host logic on CPU with gloo, world size 2:
every rank reports the slowest rank's time, and the whole-job throughput
counts every rank's bytes over that time (independent replicas, no
data-path collective)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = [12.5, 30.0][rank]                      # rank 1 is the slow replica
        m = bench.max_over_ranks(ms, world, "cpu")
        gbs = bench.job_gbs(540e6, 10, world, m)
        out[rank] = torch.tensor([m, gbs], dtype=torch.float64)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    out = torch.zeros(world, 2, dtype=torch.float64).share_memory_()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r, 0].item() == 30.0
        assert out[r, 1].item() == pytest.approx(2 * 10 * 540e6 / 0.030 / 1e9)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0
    assert bench.job_gbs(1e9, 2, 1, 1000.0) == pytest.approx(2.0)
