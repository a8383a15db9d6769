"""How many cores one B300 can simulate, per cache configuration (Table 4).

The paper's Table 4 reports the largest mesh its GPU simulator could hold in
the GPU's memory for four cache configurations (L1 sets/ways, L2 sets/ways,
with and without migration).  Here three limits are reported per
configuration: device memory (the library's own arena layout, noc_create +
noc_required_bytes, no device needed), the 65,535 tiles that 16-bit tile
indices in a flit can address -- the binding one -- and how many tiles the
fast loop holds: with one tile per thread a tile's state lives in its
thread's registers, so the register file of 148 SMs bounds the mesh; with
CTAs of up to 448 threads at 128 registers that is 148 x 448 = 66,304 tiles,
past the tile-index limit, so every mesh the indices allow whose shape cuts
into at most 148 such rectangles runs that way (the others with two tiles
per thread).  With `--run` the largest square mesh of the fast loop is found
on the GPU (a search over sides), and it and the largest mesh the tile
indices allow (255 x 257) are simulated for a few cycles.

    python -m paper_1508_03235_b300.capacity [--mem-gb G] [--run --cycles C]

Readings: the paper's L1 lines are 32 B and its L2 lines 64 B; the model has
one line size (64 B), so only the set and way counts carry over.  Rows 1 and 2
do not say whether migration was on; they are taken with migration (the
paper's full system), row 4 (without migration) as LSPD local placement.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import sys

MAX_TILES = 65535          # 16-bit tile indices in a flit
LARGEST_MESH = (255, 257)  # 65,535 tiles


def table4_rows():
    """(label, cache overrides, L2 policy) for the four rows of Table 4."""
    from . import inputs as I
    return [
        ("L1 128x4, L2 512x8", dict(l1_sets=128, l1_ways=4, l2_sets=512, l2_ways=8),
         I.POLICY_LSPD_MIGRATE),
        ("L1 128x4, L2 128x4", dict(l1_sets=128, l1_ways=4, l2_sets=128, l2_ways=4),
         I.POLICY_LSPD_MIGRATE),
        ("L1 32x2, L2 32x2, with migration", dict(l1_sets=32, l1_ways=2, l2_sets=32, l2_ways=2),
         I.POLICY_LSPD_MIGRATE),
        ("L1 32x2, L2 32x2, without migration", dict(l1_sets=32, l1_ways=2, l2_sets=32, l2_ways=2),
         I.POLICY_LSPD_LOCAL),
    ]


def params_for(w, h, cache_over, policy, seed=1):
    from . import inputs as I
    cache = I.cache_cfg()
    cache.update(cache_over)
    return I.sim_params(w, h, policy=policy, cache=cache, seed=seed)


def arena_bytes(params) -> int:
    """Device bytes of one simulation's state (the library's layout)."""
    from . import noc
    L = noc.lib()
    h = C.c_void_p()
    noc._check(L.noc_create(params["mesh_w"], params["mesh_h"], C.byref(noc.cache_struct(params)),
                            params["policy"], C.byref(noc.traffic_struct(params)), params["seed"],
                            C.byref(h)))
    try:
        return int(L.noc_required_bytes(h))
    finally:
        L.noc_destroy(h)


def capacity(cache_over, policy, mem_bytes):
    """(bytes per tile, tiles that fit mem_bytes, tiles simulable) for one row."""
    # the arena is affine in the tile count (the directory grows with the
    # private regions); measure it at two sizes and extrapolate
    a1 = arena_bytes(params_for(128, 128, cache_over, policy))
    a2 = arena_bytes(params_for(255, 257, cache_over, policy))
    n1, n2 = 128 * 128, 255 * 257
    per_tile = (a2 - a1) / (n2 - n1)
    fixed = a1 - per_tile * n1
    by_mem = int((mem_bytes - fixed) // per_tile)
    return per_tile, by_mem, min(by_mem, MAX_TILES)


def launches(side, cache_over, policy, tiles_per_thread=None) -> bool:
    """Whether a side x side mesh runs as one co-resident launch (with the
    given tiles per thread; None: the library's choice)."""
    from . import noc
    s = None
    try:
        s = noc.Sim(params_for(side, side, cache_over, policy), tiles_per_thread=tiles_per_thread)
        s.step(1)
        return True
    except noc.NocError as e:
        if e.code == 1:            # NOC_ERR_ARG: no tiling fits co-resident
            return False
        raise
    finally:
        if s is not None:
            s.close()


def largest_square(cache_over, policy, hi=255, tiles_per_thread=None) -> int:
    """The largest side whose square mesh launches (binary search)."""
    lo = 1
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if launches(mid, cache_over, policy, tiles_per_thread):
            lo = mid
        else:
            hi = mid - 1
    return lo


def run_mesh(w, h, cache_over, policy, cycles, tiles_per_thread=None):
    """Simulate a w x h mesh; (router-cycles/s, counters, tiles per thread)."""
    import time

    import torch

    from . import noc
    s = noc.Sim(params_for(w, h, cache_over, policy), tiles_per_thread=tiles_per_thread)
    s.step(50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(cycles)
    dt = time.perf_counter() - t0
    st, tpt = s.stats(), s.tiles_per_thread()
    s.close()
    return w * h * cycles / dt, st, tpt


def main(argv=None):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mem-gb", type=float, default=None,
                    help="device memory to fill (default: free memory of cuda:0, else 270)")
    ap.add_argument("--run", action="store_true")
    ap.add_argument("--cycles", type=int, default=2000)
    a = ap.parse_args(argv)
    mem = a.mem_gb * 1e9 if a.mem_gb else None
    if mem is None:
        try:
            import torch
            mem = float(torch.cuda.mem_get_info()[0]) if torch.cuda.is_available() else 270e9
        except Exception:
            mem = 270e9
    rows = []
    for label, over, pol in table4_rows():
        per_tile, by_mem, n = capacity(over, pol, mem)
        row = {"config": label, "bytes_per_tile": round(per_tile), "tiles_by_memory": by_mem,
               "tiles_by_tile_ids": MAX_TILES}
        if a.run:
            side = largest_square(over, pol, tiles_per_thread=1)
            rate1, st1, _ = run_mesh(side, side, over, pol, a.cycles, tiles_per_thread=1)
            w, h = LARGEST_MESH
            rate2, st2, tpt = run_mesh(w, h, over, pol, a.cycles)
            row.update(largest_mesh_one_tile_per_thread=f"{side}x{side}",
                       one_tile_router_cycles_per_s=rate1,
                       largest_mesh=f"{w}x{h}", max_simulated_cores=w * h, tiles_per_thread=tpt,
                       limit="16-bit tile indices", router_cycles_per_s=rate2,
                       injected=st2["injected"], ejected=st2["ejected"])
        rows.append(row)
    print(json.dumps({"device_bytes": mem, "rows": rows}, indent=1))


if __name__ == "__main__":
    main()
