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


def _sweep_worker(rank, world, port, out):
    # each rank takes its cases of the 64-case sweep with bench.shard, "runs"
    # them (a host-side cost proportional to the particle count stands in for
    # the GPU time) and the ranks combine the slowest rank's time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import casegen
        mine = bench.shard(casegen.sweep_draws(casegen.DEFAULT_SEED, 64), rank, world)
        names = [(p["alpha"], p["v0"], p["W"]) for p in mine]
        particles = sum(casegen.n_lattice(p["Lx"], p["W"], p["dx"]) for p in mine)
        t = bench.max_over_ranks(1e-6 * particles, dist)
        out[rank] = (names, particles, t)
    finally:
        dist.destroy_process_group()


def test_sweep_cases_sharded_across_two_ranks():
    import casegen
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_sweep_worker, args=(world, port, out), nprocs=world, join=True)
    every = [(p["alpha"], p["v0"], p["W"]) for p in casegen.sweep_draws(casegen.DEFAULT_SEED, 64)]
    got = [tuple(x) for x in out[0][0] + out[1][0]]
    # the shards partition the sweep: no case twice, none left out
    assert sorted(got) == sorted(every) and len(set(got)) == 64
    assert len(out[0][0]) == len(out[1][0]) == 32
    # both ranks see the slowest rank's time
    slow = max(1e-6 * out[r][1] for r in range(world))
    assert out[0][2] == out[1][2] == pytest.approx(slow)


def test_shard_partitions_for_any_world():
    items = list(range(13))
    for world in (1, 2, 3, 4, 8):
        parts = [bench.shard(items, r, world) for r in range(world)]
        assert sorted(sum(parts, [])) == items
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
