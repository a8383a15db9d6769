"""Autotuner for the CTA tiling and the router-to-thread mapping of the cycle
kernel, for single simulations and for the batch engine.

The mesh is cut into gx x gy rectangles, one CTA each (one thread per tile),
and the tiles of a rectangle are handed to its threads in one of three orders
(perimeter first, rows, columns).  Simulation results depend on neither (the
GPU tests check every tiling and order against the oracle); only the time per
simulated cycle does.  The tuner times a handful of candidate tilings in
every order on a short run of the actual configuration and keeps the fastest
pair in a JSON cache next to this file.

For the batch engine (many independent instances in work-queue launches) the
knobs are each instance's rectangle side, square or strip cut, and thread
order.  Instances are grouped by the kernel build that serves them (the
library's noc_batch_group); per group the tuner times every candidate layout
on a size-stratified sample of the workload's own descriptors and caches the
fastest under the group's key.
"""
from __future__ import annotations

import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuning_cache.json")
MAX_THREADS = 448


def key(params: dict) -> str:
    p = params
    return (f"{p['mesh_w']}x{p['mesh_h']}/pol{p['policy']}/mode{p['mode']}"
            f"/l1_{p['l1_sets']}x{p['l1_ways']}/l2_{p['l2_sets']}x{p['l2_ways']}")


def candidates(W: int, H: int, targets=(448, 384, 320, 256, 192, 160, 128, 96, 64, 32)):
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


def spread_candidates(W: int, H: int, gx: int, gy: int, max_ctas: int):
    """The other grids that cut the mesh into rectangles of the same largest
    shape as (gx, gy) -- ceil(W/gx) x ceil(H/gy) -- with at most max_ctas
    CTAs: the same warps per CTA spread over fewer or more SMs (where the cut
    falls unevenly, some rectangles are a row or column smaller).  Fewest
    CTAs first; (gx, gy) itself is not included."""
    bw, bh = -(-W // gx), -(-H // gy)
    xs = [g for g in range(1, W + 1) if -(-W // g) == bw]
    ys = [g for g in range(1, H + 1) if -(-H // g) == bh]
    out = [(a, b) for a in xs for b in ys if (a, b) != (gx, gy) and a * b <= max_ctas]
    return sorted(out, key=lambda g: (g[0] * g[1], g))


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
         verbose: bool = False, cache_path: str = CACHE):
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
        cache = (json.load(open(cache_path)) if os.path.exists(cache_path) else load_cache())
        cache[key(params)] = {"tiling": list(best[:2]), "thread_map": best[2],
                              "us_per_cycle": timings[best],
                              "timings": {f"{a}x{b}/{noc.THREAD_MAPS[m]}": v
                                          for (a, b, m), v in timings.items()},
                              "device": torch.cuda.get_device_name()}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best, timings


def spread(params: dict, cycles: int = 8000, warm: int = 2000, reps: int = 3, save: bool = True,
           verbose: bool = False, cache_path: str = CACHE):
    """Refine a cached tuning: time its tiling and every spread_candidates()
    grid of the same largest rectangle shape (up to one CTA per SM), in its
    thread order, and keep the fastest.  The grids differ by tenths of a percent, so
    each is timed longer than in tune() (8,000 cycles after 2,000, best of
    three).  Returns (best (gx, gy, order), {grid: us per cycle})."""
    import torch

    from . import noc

    cache = json.load(open(cache_path)) if os.path.exists(cache_path) else load_cache()
    entry = cache[key(params)]
    gx, gy = entry["tiling"]
    m = entry.get("thread_map", 0)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sim = noc.Sim(params, thread_map=m)
    timings = {}
    for g in [(gx, gy)] + spread_candidates(params["mesh_w"], params["mesh_h"], gx, gy, sms):
        try:
            sim.set_tiling(*g)
            dt = float("inf")
            for _ in range(reps):
                sim.reset()
                sim.step(warm)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sim.step(cycles)
                dt = min(dt, time.perf_counter() - t0)
        except noc.NocError:
            continue                       # not co-resident on this GPU
        timings[g] = 1e6 * dt / cycles
        if verbose:
            print(f"  tiling {g[0]}x{g[1]} {noc.THREAD_MAPS[m]}: {timings[g]:.3f} us/cycle", flush=True)
    sim.close()
    best = min(timings, key=timings.get)
    if save:
        entry["tiling"] = list(best)
        entry["us_per_cycle"] = timings[best]
        entry["spread_timings"] = {f"{a}x{b}/{noc.THREAD_MAPS[m]}": v for (a, b), v in timings.items()}
        cache[key(params)] = entry
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return (best[0], best[1], m), timings


# ------------------------------------------------------------------ batch engine
BATCH_SIDES = (4, 6, 8, 10, 12, 16)
GROUP_NAMES = ("interleaved 4x8", "interleaved 4x16", "interleaved 16x16", "base", "general",
               "lspd-local 4x8", "lspd-local 4x16", "lspd-local 16x16",
               "lspd-migrate 4x8", "lspd-migrate 4x16", "lspd-migrate 16x16")


def batch_key(group: int) -> str:
    return f"batch/group{group}"


def cached_batch_layout(group: int):
    """The tuned (rect side, strips, thread order) of a kernel-variant group,
    or None."""
    t = load_cache().get(batch_key(group))
    return (t["rect"], bool(t["strips"]), t["thread_map"]) if t else None


def stratified_sample(params_list, idx, k):
    """k of the instances idx, spread evenly over their sizes."""
    order = sorted(idx, key=lambda i: (params_list[i]["mesh_w"] * params_list[i]["mesh_h"], i))
    if len(order) <= k:
        return order
    return [order[(j * len(order)) // k] for j in range(k)]


def batch_candidates(sides=BATCH_SIDES, maps=(0, 1, 2)):
    return [(side, strips, m) for side in sides for strips in (False, True) for m in maps]


def tune_batch(params_list, cycles: int = 3000, sample: int = 48, reps: int = 2, save: bool = True,
               cache_path: str = CACHE, verbose: bool = False):
    """Per kernel-variant group of params_list: time every candidate layout
    (batch_candidates) on a sample of the group's instances, `cycles` each,
    best of `reps` runs after a warm-up run; cache the fastest.  Returns
    {group: (best layout, {layout: seconds})}."""
    import torch

    from . import noc

    groups = noc.batch_groups(params_list)
    out = {}
    for g in sorted(set(groups)):
        idx = stratified_sample(params_list, [i for i, x in enumerate(groups) if x == g], sample)
        pts = [params_list[i] for i in idx]
        timings = {}
        for side, strips, m in batch_candidates():
            b = noc.Batch(pts, cycles, collect_hash=False, rect=side, strips=strips, thread_map=m)
            try:
                b.run()
                dt = float("inf")
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    b.run()
                    dt = min(dt, time.perf_counter() - t0)
            except noc.NocError:
                continue                   # an instance does not fit at this side
            finally:
                b.close()
            timings[(side, strips, m)] = dt
            if verbose:
                print(f"  group {GROUP_NAMES[g]}: side {side} {'strips' if strips else 'squares'} "
                      f"{noc.THREAD_MAPS[m]}: {1e3 * dt:.1f} ms", flush=True)
        best = min(timings, key=timings.get)
        out[g] = (best, timings)
        if save:
            cache = load_cache() if cache_path == CACHE else (
                json.load(open(cache_path)) if os.path.exists(cache_path) else load_cache())
            cache[batch_key(g)] = {
                "group": GROUP_NAMES[g], "rect": best[0], "strips": int(best[1]), "thread_map": best[2],
                "sample_instances": len(pts), "cycles": cycles, "seconds": timings[best],
                "sims_per_s_sample": len(pts) / timings[best],
                "timings_ms": {f"{a}/{'strips' if b_ else 'squares'}/{noc.THREAD_MAPS[c]}": 1e3 * v
                               for (a, b_, c), v in timings.items()},
                "device": torch.cuda.get_device_name()}
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
    return out


if __name__ == "__main__":
    import argparse
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import tune as T
    ap = argparse.ArgumentParser(description="autotune the cycle kernel's layouts")
    ap.add_argument("--broad", action="store_true", help="every rectangle shape (single simulations)")
    ap.add_argument("--batch", action="store_true",
                    help="tune the batch engine on the 512-instance design-point workload")
    ap.add_argument("--spread", action="store_true",
                    help="refine the cached single-simulation tilings over more CTAs of the same shape")
    ap.add_argument("--out", default=CACHE, help="cache file to update")
    a = ap.parse_args()
    if a.spread:
        for name, p in (("mesh208", I.mesh_208(10)), ("mesh64", I.mesh_64(1)),
                        ("mesh8", I.MESH_8["params"])):
            print(name, flush=True)
            b, t = T.spread(p, verbose=True, cache_path=a.out)
            print(f"  best {b}", flush=True)
    elif a.batch:
        pts = I.batch_design_points(512, seed=0)
        for p in pts:
            p.pop("design")
        for g, (best, t) in T.tune_batch(pts, cache_path=a.out, verbose=True).items():
            print(f"group {T.GROUP_NAMES[g]}: best {best}", flush=True)
    else:
        for name, p in (("mesh208", I.mesh_208(10)), ("mesh64", I.mesh_64(1)),
                        ("mesh8", I.MESH_8["params"])):
            print(name, flush=True)
            b, t = T.tune(p, broad=a.broad, verbose=not a.broad, cache_path=a.out)
            if a.broad:
                for k in sorted(t, key=t.get)[:10]:
                    print(f"  {k[0]}x{k[1]} order {k[2]}: {t[k]:.3f} us/cycle", flush=True)
            print(f"  best {b}", flush=True)
