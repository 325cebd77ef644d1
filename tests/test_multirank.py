"""The benchmark's multi-rank logic on two CPU ranks (gloo): replicas run
independently, the job's time is the slowest rank's, and the whole-job value
counts every rank's node updates.  No GPU and no data-path collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench.dist_env()
        assert (ws, r) == (world, rank)
        my_ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
        slowest = bench.max_over_ranks(my_ms)
        out[rank] = (slowest, bench.replica_throughput(ws, 524288, 20, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_timing_and_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, value = res[rank]
        assert slowest == 150.0
        assert value == pytest.approx(2 * 524288 * 20 / 0.150 / 1e6)


def test_single_process_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(1, 1000, 10, 2.0) == pytest.approx(5.0)
    assert torch.tensor([1.0]).device.type == "cpu"

