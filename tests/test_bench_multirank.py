"""Replica aggregation of bench.py across ranks (world size 2, gloo, CPU):
the job's time is the slowest rank's and its work the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, units = bench.reduce_over_ranks(100.0 * (rank + 1), 10 * (rank + 1))
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == (200.0, 30.0)


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7.0)
