"""Replicas on several processes (bench.py under torchrun): the job's time is
the slowest rank's and its throughput counts every replica's work.  Run here as
two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    dist.barrier()
    out[rank] = (slowest, bench.replica_value(1000.0, 10, world, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    slowest, value = out[0]
    assert slowest == 150.0
    assert value == pytest.approx(2 * 1000.0 * 10 / 0.150)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_value(10.0, 4, 1, 2.0) == pytest.approx(20000.0)
