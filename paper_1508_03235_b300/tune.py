"""Autotuner for the CTA tiling and the router-to-thread mapping of the cycle
kernel.

The mesh is cut into gx x gy rectangles, one CTA each (one thread per tile),
and the tiles of a rectangle are handed to its threads in one of three orders
(perimeter first, rows, columns).  Simulation results depend on neither (the
GPU tests check every tiling and order against the oracle); only the time per
simulated cycle does.  The tuner times a handful of candidate tilings in
every order on a short run of the actual configuration and keeps the fastest
pair in a JSON cache next to this file.
"""
from __future__ import annotations

import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuning_cache.json")
MAX_THREADS = 384


def key(params: dict) -> str:
    p = params
    return (f"{p['mesh_w']}x{p['mesh_h']}/pol{p['policy']}/mode{p['mode']}"
            f"/l1_{p['l1_sets']}x{p['l1_ways']}/l2_{p['l2_sets']}x{p['l2_ways']}")


def candidates(W: int, H: int, targets=(384, 320, 256, 192, 160, 128, 96, 64, 32)):
    """For each rectangle-size target, the grid with the fewest CTAs whose
    rectangles hold at most that many tiles, preferring aspect ratios <= 2.5."""
    out = []
    for target in targets:
        best = None
        for gy in range(1, H + 1):
            bh = -(-H // gy)
            for gx in range(1, W + 1):
                bw = -(-W // gx)
                if bw * bh > min(target, MAX_THREADS):
                    continue
                skew = abs(math.log(bw / bh))
                k = (skew > math.log(2.5), gx * gy, skew)
                if best is None or k < best[0]:
                    best = (k, (gx, gy))
                break                      # larger gx only adds CTAs for this gy
        if best and best[1] not in out:
            out.append(best[1])
    return out


def broad_candidates(W: int, H: int, lo: int = 48, hi: int = MAX_THREADS):
    """Every rectangle shape of lo..hi tiles the mesh can be cut into, each
    with the fewest CTAs that give it, largest rectangles first."""
    best = {}
    for gy in range(1, H + 1):
        for gx in range(1, W + 1):
            bw, bh = -(-W // gx), -(-H // gy)
            if not lo <= bw * bh <= hi:
                continue
            if (bw, bh) not in best or gx * gy < best[(bw, bh)][0] * best[(bw, bh)][1]:
                best[(bw, bh)] = (gx, gy)
    return sorted(best.values(), key=lambda g: (-(-(-W // g[0]) * -(-H // g[1])), g))


def load_cache() -> dict:
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            return json.load(f)
    return {}


def cached_tiling(params: dict):
    t = load_cache().get(key(params))
    return tuple(t["tiling"]) if t else None


def cached_thread_map(params: dict):
    """The tuned tile-to-thread order, or None (the library default)."""
    t = load_cache().get(key(params))
    return t.get("thread_map", 0) if t else None


def tune(params: dict, cycles: int = 2000, warm: int = 200, max_cands: int = 10,
         maps=(0, 1, 2), reps: int = 2, broad: bool = False, save: bool = True,
         verbose: bool = False):
    """Time candidate tilings in each tile-to-thread order (the best of `reps`
    timed runs each); return (best (gx, gy, order), {(gx, gy, order): us per
    cycle}).  With `broad`, every rectangle shape of broad_candidates() is
    tried instead of one grid per size target."""
    import torch

    from . import noc

    sim = noc.Sim(params)
    timings = {}
    cands = (broad_candidates(params["mesh_w"], params["mesh_h"]) if broad
             else candidates(params["mesh_w"], params["mesh_h"])[:max_cands])
    for gx, gy in cands:
        for m in maps:
            try:
                sim.set_tiling(gx, gy)
                sim.set_thread_map(m)
                dt = float("inf")
                for _ in range(reps):
                    sim.reset()
                    sim.step(warm)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    sim.step(cycles)
                    dt = min(dt, time.perf_counter() - t0)
            except noc.NocError:
                break                      # not co-resident on this GPU
            timings[(gx, gy, m)] = 1e6 * dt / cycles
            if verbose:
                print(f"  tiling {gx}x{gy} {noc.THREAD_MAPS[m]}: {timings[(gx, gy, m)]:.2f} us/cycle",
                      flush=True)
    sim.close()
    best = min(timings, key=timings.get)
    if save:
        cache = load_cache()
        cache[key(params)] = {"tiling": list(best[:2]), "thread_map": best[2],
                              "us_per_cycle": timings[best],
                              "timings": {f"{a}x{b}/{noc.THREAD_MAPS[m]}": v
                                          for (a, b, m), v in timings.items()},
                              "device": torch.cuda.get_device_name()}
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best, timings


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300.tune import tune as _tune
    broad = "--broad" in sys.argv
    for name, p in (("mesh208", I.mesh_208(10)), ("mesh64", I.mesh_64(1)),
                    ("mesh8", I.MESH_8["params"])):
        print(name, flush=True)
        b, t = _tune(p, broad=broad, verbose=not broad)
        if broad:
            for k in sorted(t, key=t.get)[:10]:
                print(f"  {k[0]}x{k[1]} order {k[2]}: {t[k]:.3f} us/cycle", flush=True)
        print(f"  best {b}", flush=True)
