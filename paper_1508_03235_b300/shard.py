"""Splitting a batch of independent simulations over ranks (one process per
GPU) and collecting the per-instance results on rank 0.

The batch workload's instances share nothing, so a multi-GPU run needs no
exchange on the data path: each rank simulates its own share with the batch
engine, and only the small per-instance results travel, once, at the end
(torch.distributed.all_gather_object: NCCL between GPUs, gloo in the CPU
tests).  The share of each rank is chosen by cost (tiles x cycles), largest
first onto the least-loaded rank, so the ranks finish at about the same time.
"""
from __future__ import annotations


def instance_cost(params: dict, cycles: int) -> int:
    """Work of one instance: router-cycles."""
    return params["mesh_w"] * params["mesh_h"] * int(cycles)


def partition_by_cost(costs, world: int):
    """Longest-processing-time-first split of instance indices over `world`
    ranks: each instance, most expensive first (ties by index), goes to the
    rank with the least work so far (ties by rank).  Every index lands on
    exactly one rank; each rank's list is in ascending index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(local: dict, n: int, world: int):
    """All ranks' {instance index: result} merged on every rank (collective:
    every rank must call it).  Raises if an instance is missing or was run by
    two ranks."""
    if world == 1:
        merged = dict(local)
    else:
        import torch.distributed as dist
        got = [None] * world
        dist.all_gather_object(got, local)
        merged = {}
        for part in got:
            for i, v in part.items():
                if i in merged:
                    raise RuntimeError(f"instance {i} was run by two ranks")
                merged[i] = v
    missing = [i for i in range(n) if i not in merged]
    if missing:
        raise RuntimeError(f"instances never run: {missing[:8]}")
    return merged
