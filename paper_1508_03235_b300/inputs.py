"""Seeded workload parameters shared by the CUDA path and the oracle.

This module holds parameter sets and the design-point sampler only: no step
of the simulated model.  The reference stream itself is drawn inside each
simulator from a counter-based Philox4x64-10 keyed by (seed, core, ref), so the
two implementations see identical inputs without sharing code.

The paper's workloads are Multi2sim address traces of matmul and SPEC OMP 2001
programs (Sec. 6.2.3, Sec. 8); those traces are not available, and these
synthetic mixes stand in for them:

* MESH_8   -- 8x8 mesh, one reference per 10 cycles, 30% writes, 70% of
              references to a 16 KB private working set, 20% uniform over a
              4 MB shared region, 10% uniform over 1 GB; 20,000 cycles, seed 1.
* MESH_64  -- 64x64 mesh, same caches, one reference per 4 cycles, 40% of
              shared references go to lines homed on the 4x4 tiles nearest the
              mesh centre; 100,000 cycles, seeds 1-4.
* MESH_208 -- 208x208 mesh (43,264 tiles, the paper's largest scale), 512 KB
              16-way L2 slices, the MESH_8 mix, one reference per
              {40, 20, 10, 5, 2} cycles, 50,000 cycles, seed 7.
* batch_design_points -- independent instances of mixed size, load, address
              mix and L2 policy (sides 8..128, Dirichlet(2,2,1) fractions).
"""
from __future__ import annotations

import numpy as np

Q16 = 65536

POLICY_INTERLEAVED = 0
POLICY_LSPD_LOCAL = 1
POLICY_LSPD_MIGRATE = 2
POLICY_NAMES = {0: "interleaved", 1: "lspd-local", 2: "lspd-migrate"}

MODE_CACHE = 0
MODE_NETWORK = 1
MODE_TRACE = 2

LINE_BYTES = 64


def q16(frac: float) -> int:
    """A fraction in [0, 1] as a 16-bit fixed-point threshold."""
    return int(round(frac * Q16))


def cache_cfg(l1_kb=32, l1_ways=4, l2_kb=256, l2_ways=8, **over):
    """Cache geometry and latencies; 64 B lines."""
    cfg = dict(
        l1_sets=l1_kb * 1024 // LINE_BYTES // l1_ways,
        l1_ways=l1_ways,
        l2_sets=l2_kb * 1024 // LINE_BYTES // l2_ways,
        l2_ways=l2_ways,
        l1_miss_cycles=4,
        mem_latency=100,
        mig_window=10,
        mig_threshold=6,
        core_q=8,
        svc_q=256,
        mem_q=128,
        fwd_entries=4,
        packet_mode=0,
        rob_entries=8,
        dir_central=0,
        dir_tile=0,
        l1_write_back=0,
        age_mode=0,
    )
    cfg.update(over)
    return cfg


def traffic(period=10, write=0.30, priv=0.70, shared=0.20, hot=0.0, hot_side=0,
            priv_kb=16, shared_mb=4, remote_gb=1, mode=MODE_CACHE):
    """Reference-stream parameters (fractions are quantised to q16)."""
    return dict(
        mode=mode,
        period=period,
        write_q16=q16(write),
        priv_q16=q16(priv),
        shared_q16=q16(shared),
        hot_q16=q16(hot),
        hot_side=hot_side,
        priv_lines=priv_kb * 1024 // LINE_BYTES,
        shared_lines=shared_mb * 1024 * 1024 // LINE_BYTES,
        remote_lines=remote_gb * 1024 * 1024 * 1024 // LINE_BYTES,
    )


def sim_params(w, h, policy=POLICY_INTERLEAVED, cache=None, traf=None, seed=1, stream=0):
    """One simulation's full parameter set as a flat dict."""
    p = dict(mesh_w=w, mesh_h=h, policy=policy, seed=seed, stream=stream)
    p.update(cache if cache is not None else cache_cfg())
    p.update(traf if traf is not None else traffic())
    return p


# --- the named workloads ---------------------------------------------------
MESH_8 = dict(params=sim_params(8, 8, seed=1), cycles=20_000)
MESH_64_SEEDS = (1, 2, 3, 4)
MESH_64_CYCLES = 100_000
MESH_208_PERIODS = (40, 20, 10, 5, 2)
MESH_208_CYCLES = 50_000
MESH_208_SEED = 7


def mesh_64(seed=1):
    return sim_params(64, 64, seed=seed,
                      traf=traffic(period=4, hot=0.40, hot_side=4),
                      cache=cache_cfg(svc_q=1024))


def mesh_208(period=10, seed=MESH_208_SEED):
    return sim_params(208, 208, seed=seed,
                      cache=cache_cfg(l2_kb=512, l2_ways=16, svc_q=1024),
                      traf=traffic(period=period))


# --- batch design points -----------------------------------------------------
WS_KB_CHOICES = (4, 8, 16, 32, 64)


def batch_design_points(n=512, seed=0, sides=tuple(range(8, 129, 8)), period_lo=2,
                        period_hi=40, policies=(0, 1, 2), write_lo=0.1, write_hi=0.5):
    """Independent instances: side U{8,16,..,128}, period U{2..40}, address
    fractions Dirichlet(2,2,1) (private, shared, remote), policy uniform,
    write fraction U[0.1,0.5], private working set from {4..64} KB.
    Instance i has seed i+1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.choice(sides))
        period = int(rng.integers(period_lo, period_hi + 1))
        fr = rng.dirichlet((2.0, 2.0, 1.0))
        pol = int(rng.choice(policies))
        write = float(rng.uniform(write_lo, write_hi))
        ws_kb = int(rng.choice(WS_KB_CHOICES))
        pq, sq = q16(fr[0]), q16(fr[1])
        if pq + sq > Q16:
            sq = Q16 - pq
        traf = traffic(period=period, write=0.0, priv=0.0, shared=0.0, priv_kb=ws_kb)
        traf.update(write_q16=q16(write), priv_q16=pq, shared_q16=sq)
        p = sim_params(side, side, policy=pol, seed=i + 1, traf=traf,
                       cache=cache_cfg(svc_q=512))
        p["design"] = dict(side=side, period=period, priv=pq / Q16, shared=sq / Q16,
                           remote=1.0 - (pq + sq) / Q16, write=write, ws_kb=ws_kb, policy=pol)
        out.append(p)
    return out
