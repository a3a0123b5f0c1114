"""The multi-GPU path of the benchmark is replicas only: each rank runs its
own system and the only collective is the MAX over ranks of the step time.
Checked here with two gloo ranks on the CPU (no GPU involved)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [3.0, 5.0][rank]          # the ranks' own step times
        ms = bench.replica_time(local_ms, dist, "cpu")
        out[rank] = (ms, bench.replica_value(ms, 1000, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 5.0
        assert value == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_is_its_own_time():
    assert bench.replica_time(4.0) == 4.0
    assert bench.replica_value(4.0, 100_000, 1) == pytest.approx(100_000 / 4e-3)
