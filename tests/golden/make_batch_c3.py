"""Write tests/golden/batch_c3.json: the oracle's results for every instance
of the 512-instance batch workload (sides 8..128, periods 2..40,
Dirichlet(2,2,1) address mixes, all three L2 policies, seeds 1..512), 20,000
cycles each.

Calls only the oracle (oracle/) and the seeded workload parameters
(paper_1508_03235_b300/inputs.py).  Per instance: every counter, the full
state hash, and a SHA-256 digest (first 16 hex digits) of each latency
histogram's 1,025 little-endian uint64 bins.  The GPU test
tests/test_gpu_batch_c3.py runs the whole batch through libnoc.so in the
benchmark's configuration and compares every instance with these records.
One oracle process per host core (about 75 core-minutes in all).

    python tests/golden/make_batch_c3.py [--jobs N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "batch_c3.json")
N, CYCLES, SEED = 512, 20_000, 0


def hist_digest(h) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest()[:16]


def run_job(job):
    i, params = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle
    o = oracle.OracleSim(params)
    o.step(CYCLES)
    rec = dict(stats=o.stats(), state_hash=str(o.state_hash()),
               hist_sha=[hist_digest(o.hist(w)) for w in (0, 1)])
    o.close()
    return i, rec


def points():
    from paper_1508_03235_b300 import inputs as I
    pts = I.batch_design_points(N, seed=SEED)
    for p in pts:
        p.pop("design")
    return pts


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    from oracle import oracle
    oracle.build()
    pts = points()
    jobs = sorted(enumerate(pts), key=lambda j: -j[1]["mesh_w"] * j[1]["mesh_h"])
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        res = dict(pool.map(run_job, jobs, chunksize=1))
    doc = {"generator": "tests/golden/make_batch_c3.py (the serial oracle, oracle/noc_oracle.c)",
           "instances": N, "cycles": CYCLES, "design_seed": SEED,
           "records": [res[i] for i in range(N)]}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, separators=(",", ":"), sort_keys=True)
        fh.write("\n")
    print(f"wrote {OUT} in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()
