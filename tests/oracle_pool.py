"""Oracle runs spread over the host's cores (test infrastructure).

A `spawn` process pool, so it is safe to start after the parent has touched
the GPU; each worker loads the serial oracle and returns one instance's
counters, full state hash and both latency histograms.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_one(job):
    params, cycles = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle
    o = oracle.OracleSim(params)
    o.step(cycles)
    out = (o.stats(), o.state_hash(), o.hist(0), o.hist(1))
    o.close()
    return out


def run_many(params_list, cycles, procs=None):
    """Results in the order of params_list; the largest instances start first."""
    import multiprocessing as mp
    order = sorted(range(len(params_list)),
                   key=lambda i: -params_list[i]["mesh_w"] * params_list[i]["mesh_h"])
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs or os.cpu_count() or 1) as pool:
        res = pool.map(run_one, [(params_list[i], cycles) for i in order], chunksize=1)
    out = [None] * len(params_list)
    for i, r in zip(order, res):
        out[i] = r
    return out
