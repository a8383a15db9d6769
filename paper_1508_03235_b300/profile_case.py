"""A short, warmed-up run of a named workload, sized for one profiler capture.

    python -m paper_1508_03235_b300.profile_case --mesh 208 --warm 2000 --cycles 1024

runs `--warm` cycles (one or more cycle-kernel launches), then exactly one
launch of `--cycles` cycles, and prints the cycle count.  Capture that last
launch with `-k regex:run_kernel -s <launches of the warm-up> -c 1`; the number
of warm-up launches is printed as well.  The 208x208 state is about 1.6 GB.
With `--phases` the timed launch runs on the build with per-phase clock reads
(noc_set_phase_profile) and the SM clocks per warp-cycle of each phase are
printed.

    python -m paper_1508_03235_b300.profile_case --case surrogate

runs the fused surrogate inference (mlp_infer) three times on a batch of 4096
design points: capture `-k regex:infer_kernel -s 2 -c 1`.

    python -m paper_1508_03235_b300.profile_case --case batch --instances 64 --batch-cycles 2000

runs the first `--instances` design points of the batch workload for
`--batch-cycles` cycles through the batch engine (the autotuner's layout per
kernel-variant group): one work-queue launch per group; capture
`-k regex:batch_kernel -c 1`.
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
    ap.add_argument("--case", default="cycle", choices=("cycle", "surrogate", "batch"))
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--batch-cycles", type=int, default=2000)
    ap.add_argument("--phases", action="store_true",
                    help="run the timed launch on the build with per-phase clock reads and print them")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    if a.case == "surrogate":
        from paper_1508_03235_b300 import surrogate as S
        net = S.MLP(seed=0, max_batch=4096)
        xb = torch.rand(4096, S.DIMS[0], device="cuda").to(torch.bfloat16)
        y = torch.empty(4096, S.DIMS[-1], device="cuda")
        for _ in range(3):
            net.infer(xb, out=y)
        torch.cuda.synchronize()
        print(f"surrogate {list(S.DIMS)}: 3 fused inferences of 4096 points, status {S.gemm_status()}")
        return
    if a.case == "batch":
        from paper_1508_03235_b300 import inputs as I
        from paper_1508_03235_b300 import noc
        pts = I.batch_design_points(512, seed=0)[: a.instances]
        for p in pts:
            p.pop("design")
        b = noc.Batch(pts, a.batch_cycles, collect_hash=False)     # the tuned layouts
        b.run()
        torch.cuda.synchronize()
        tiles = sum(p["mesh_w"] * p["mesh_h"] for p in pts)
        print(f"batch of {len(pts)} instances ({tiles} tiles) x {a.batch_cycles} cycles done")
        return

    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc, tune
    p = {8: I.MESH_8["params"], 64: I.mesh_64(1), 208: I.mesh_208(a.period)}[a.mesh]
    s = noc.Sim(p, tiling=tune.cached_tiling(p), thread_map=tune.cached_thread_map(p))
    s.kernel_time(True)
    s.step(a.warm)
    _, warm_launches = s.kernel_time(True)
    if a.phases:
        s.set_phase_profile(True)
    s.step(a.cycles)
    torch.cuda.synchronize()
    ms, n = s.kernel_time(False)
    print(f"mesh {a.mesh}x{a.mesh} tiling {s.tiling()} warm-up launches {warm_launches} "
          f"then {n} launch of {a.cycles} cycles ({ms:.3f} ms); cycle {s.stats()['cycle']}")
    if a.phases:
        prof = s.phase_profile()
        print("SM clocks per warp-cycle: " + ", ".join(f"{k} {prof[k]:.0f}" for k in s.PHASES)
              + f" ({prof['warp_cycles']} warp-cycles)")


if __name__ == "__main__":
    main()
