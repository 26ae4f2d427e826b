"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own replica, the slowest rank's time decides, and the whole-job
value counts every rank's iterations."""

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


def _worker(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_timing(local_ms[rank], 100, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    world, port = 2, _free_port()
    local_ms = [3.0, 5.0]  # rank 1 is slower
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, local_ms, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == pytest.approx(5.0 / 100)
        assert value == pytest.approx(2 * 100 / 5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_timing(7.0, 70, 1, torch.device("cpu"))
    assert ms == pytest.approx(0.1) and value == pytest.approx(10_000.0)
