"""A short, warmed-up run of a named workload, sized for one profiler capture.

    python -m paper_1508_03235_b300.profile_case --mesh 208 --warm 2000 --cycles 1024

runs `--warm` cycles (one or more cycle-kernel launches), then exactly one
launch of `--cycles` cycles, and prints the cycle count.  Capture that last
launch with `-k regex:run_kernel -s <launches of the warm-up> -c 1`; the number
of warm-up launches is printed as well.  The 208x208 state is about 1.6 GB.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=208, choices=(8, 64, 208))
    ap.add_argument("--period", type=int, default=10)
    ap.add_argument("--warm", type=int, default=2000)
    ap.add_argument("--cycles", type=int, default=1024)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc, tune
    p = {8: I.MESH_8["params"], 64: I.mesh_64(1), 208: I.mesh_208(a.period)}[a.mesh]
    s = noc.Sim(p, tiling=tune.cached_tiling(p), thread_map=tune.cached_thread_map(p))
    s.kernel_time(True)
    s.step(a.warm)
    _, warm_launches = s.kernel_time(True)
    s.step(a.cycles)
    torch.cuda.synchronize()
    ms, n = s.kernel_time(False)
    print(f"mesh {a.mesh}x{a.mesh} tiling {s.tiling()} warm-up launches {warm_launches} "
          f"then {n} launch of {a.cycles} cycles ({ms:.3f} ms); cycle {s.stats()['cycle']}")


if __name__ == "__main__":
    main()
