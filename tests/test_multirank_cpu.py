"""Host-side logic of the multi-GPU bench on CPU: two gloo ranks, each with
its own replica timing, combine to the maximum over ranks and the aggregate
particle-steps/s (the path itself does not shard: replicas only)."""
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


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist)
        v = bench.aggregate_value(world, 1000, 10, t)
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_aggregate(world):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    times = [12.5, 20.0]
    mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 20.0
        assert v == pytest.approx(world * 1000 * 10 / 0.020)


def test_single_rank_passthrough():
    assert bench.max_over_ranks(7.25, None) == 7.25
    assert bench.aggregate_value(1, 1_125_000, 200, 42.0) == pytest.approx(1_125_000 * 200 / 0.042)
