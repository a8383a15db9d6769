"""Splitting the batch workload's independent instances over ranks: the cost
partition covers every instance once and balances the work, and two gloo
ranks that each simulate their share (with the oracle, on the CPU) gather a
complete set of per-instance results equal to simulating every instance in
one process."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1508_03235_b300 import inputs as I
from paper_1508_03235_b300 import shard


def test_partition_covers_every_instance_once_and_balances():
    pts = I.batch_design_points(512, seed=0)
    costs = [shard.instance_cost(p, 20_000) for p in pts]
    for world in (1, 2, 3, 8):
        parts = shard.partition_by_cost(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: no rank exceeds the mean by more than the largest single instance
        assert max(loads) - sum(loads) / world <= max(costs)
    assert shard.partition_by_cost([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]
    with pytest.raises(ValueError):
        shard.partition_by_cost([1], 0)


def test_gather_single_rank_checks_completeness():
    assert shard.gather_results({0: 1, 1: 2}, 2, 1) == {0: 1, 1: 2}
    with pytest.raises(RuntimeError):
        shard.gather_results({0: 1}, 2, 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def small_points():
    pts = I.batch_design_points(10, seed=5, sides=(4, 6, 8, 10), period_lo=3, period_hi=9)
    for p in pts:
        p.pop("design")
    return pts


def _one(p, cycles):
    from oracle import oracle
    o = oracle.OracleSim(p)
    o.step(cycles)
    out = (o.stats()["ejected"], o.stats()["l2lat_sum"], o.state_hash())
    o.close()
    return out


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts, cycles = small_points(), 300
    parts = shard.partition_by_cost([shard.instance_cost(p, cycles) for p in pts], world)
    local = {i: _one(pts[i], cycles) for i in parts[rank]}
    merged = shard.gather_results(local, len(pts), world)
    out[rank] = (parts[rank], merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_and_gather_real_instances(oracle_mod):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert sorted(out[0][0] + out[1][0]) == list(range(10)) and out[0][0] and out[1][0]
    assert out[0][1] == out[1][1]
    pts = small_points()
    assert out[0][1] == {i: _one(p, 300) for i, p in enumerate(pts)}
