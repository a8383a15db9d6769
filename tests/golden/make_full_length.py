"""Write tests/golden/full_length.json: the oracle's results on the named
workloads at their full configured lengths.

Calls only the oracle (oracle/) and the seeded workload parameters
(paper_1508_03235_b300/inputs.py); nothing from the CUDA path.  The GPU parity
tests (tests/test_gpu_full_length.py) run the same workloads through libnoc.so
and compare with these records, bit for bit, at every checkpoint:

* the 64x64 hotspot mesh, seeds 1-4, 100,000 cycles (checkpoints 2,000,
  20,000 and 100,000);
* the 208x208 mesh at each injection period {40, 20, 10, 5, 2}, seed 7,
  50,000 cycles (checkpoints 2,000, 10,000 and 50,000).

Each checkpoint holds every counter, the dynamic and full state hashes, and
both latency histograms (as {bin: count} of the non-empty bins).  The jobs run
in parallel, one oracle process per job (about 6 minutes over 8 cores).

    python tests/golden/make_full_length.py [--jobs N]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "full_length.json")


def workloads():
    from paper_1508_03235_b300 import inputs as I
    out = []
    for seed in I.MESH_64_SEEDS:
        out.append((f"mesh64_hotspot_seed{seed}", I.mesh_64(seed), (2_000, 20_000, I.MESH_64_CYCLES)))
    for period in I.MESH_208_PERIODS:
        out.append((f"mesh208_period{period}", I.mesh_208(period), (2_000, 10_000, I.MESH_208_CYCLES)))
    return out


def run_job(job):
    name, params, checkpoints = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle
    o = oracle.OracleSim(params)
    recs, done = [], 0
    for c in checkpoints:
        t0 = time.perf_counter()
        o.step(c - done)
        dt = time.perf_counter() - t0
        done = c
        recs.append(dict(
            cycle=c, stats=o.stats(), dyn_hash=str(o.dyn_hash()), state_hash=str(o.state_hash()),
            hist=[{str(i): int(v) for i, v in enumerate(o.hist(w)) if v} for w in (0, 1)],
            oracle_seconds=round(dt, 2)))
    o.close()
    return name, dict(params=params, checkpoints=recs)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    from oracle import oracle
    oracle.build()
    jobs = workloads()
    jobs.sort(key=lambda j: -j[1]["mesh_w"] * j[1]["mesh_h"] * j[2][-1])
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        res = dict(pool.map(run_job, jobs, chunksize=1))
    doc = {"generator": "tests/golden/make_full_length.py (the serial oracle, oracle/noc_oracle.c)",
           "workloads": {name: res[name] for name, _, _ in workloads()}}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(f"wrote {OUT} in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()
