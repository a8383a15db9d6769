"""Benchmark: simulated router-cycles/s on the 208x208 mesh (43,264 tiles).

One step = the paper's largest configuration swept over injection periods
{40, 20, 10, 5, 2}: for each period, reset the simulation to cycle 0 and run
50,000 cycles (five persistent cooperative launches in all).  Timed on the
device with CUDA events on the simulator's stream; the state touched per run
(1.4 GB of L2 tags plus L1s, queues and links) is larger than the GPU's L2.

`--impl reference` times the oracle (the serial C simulator) on the host cores
for the same metric on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1508_03235_b300 import inputs as I  # noqa: E402

METRIC = "router-cycles/s at 208x208 mesh (bit-exact simulation)"
UNIT = "router-cycles/s"
PERIODS = I.MESH_208_PERIODS
CYCLES = I.MESH_208_CYCLES
TILES = 208 * 208


def workload_config(extra=None):
    cfg = {"workload": "mesh208_period_sweep", "mesh": "208x208", "tiles": TILES,
           "periods": list(PERIODS), "cycles_per_run": CYCLES, "runs_per_step": len(PERIODS),
           "seed": I.MESH_208_SEED, "l1": "32KB 4-way", "l2": "512KB 16-way per tile",
           "l2_policy": "interleaved (home = line mod N)",
           "traffic": "Philox stream: 30% writes, 70/20/10 private 16KB/shared 4MB/remote 1GB",
           "l2_flush": "inputs larger than L2: 1.4 GB of L2 tags plus L1/queue/link state per run"}
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"noc_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path).read().splitlines()[1:]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def algorithmic_bytes(stats_delta, router_cycles, p):
    """State bytes a cycle-stepped simulator must touch: per router-cycle the
    four in-link and four out-link slots (8 x 16 B) and the tile's 13-word
    core record read and written (2 x 52 B); per L1 lookup or fill one L1 set
    read and written; per L2 access (lookup, install, write-through) one L2
    set read and written; per injected flit one 16 B queue push and pop."""
    l1set = 4 * p["l1_ways"]
    l2set = 4 * p["l2_ways"]
    d = stats_delta
    l1_ops = d["l1_hit"] + d["l1_miss"] + d["l2lat_cnt"]          # lookups + fills
    l2_ops = d["l2_hit"] + d["l2_miss"] + d["wt_hit"] + d["mem_write"] + d["mem_req"]
    return (router_cycles * (8 * 16 + 2 * 52) + l1_ops * 2 * l1set + l2_ops * 2 * l2set
            + d["injected"] * 2 * 16)


KERNEL_SOURCES = ("noc_model.cuh", "noc_kernel.cuh", "noc_internal.h", "noc_run_variant.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "run_kernel_mesh208_traffic.md")


def kernel_sources_sha256() -> str:
    """sha256 of the cycle kernel's sources with comments and blank space
    removed (so editing a comment does not orphan a capture)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1508_03235_b300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def measured_traffic(cycles_per_launch):
    """DRAM bytes (read + write) per cycle-kernel launch, scaled from the
    committed ncu capture of the same kernel sources (by cycles per launch);
    None when there is no capture or the kernel changed since it was taken."""
    import re
    if not os.path.exists(TRAFFIC_FILE):
        return None
    text = open(TRAFFIC_FILE).read()
    sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    per = re.search(r"dram_bytes_per_cycle:\s*([0-9.eE+]+)", text)
    if not sha or not per or sha.group(1) != kernel_sources_sha256():
        return None
    return float(per.group(1)) * cycles_per_launch


# --------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1508_03235_b300 import noc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1508_03235_b300 import tune
    stream = torch.cuda.current_stream()
    # tiling: the autotuner's cached choice for this configuration, if any
    sims = [noc.Sim(I.mesh_208(P), stream=stream, tiling=tune.cached_tiling(I.mesh_208(P)),
                    thread_map=tune.cached_thread_map(I.mesh_208(P)))
            for P in PERIODS]
    tiling = sims[0].tiling()
    cycles = args.cycles

    def one_step():
        for s in sims:
            s.reset()
            s.step_async(cycles)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    for s in sims:
        s.sync()
    tiling = sims[0].tiling()
    launches0 = sum(s.launches for s in sims)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for s in sims:
        s.kernel_time(True)               # events around every cycle-kernel launch
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        one_step()
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    for s in sims:
        s.sync()
    ms = t_start.elapsed_time(t_end)
    gpu_launches = sum(s.launches for s in sims) - launches0
    rc_per_rank = args.steps * len(PERIODS) * TILES * cycles
    ms, value = replica_throughput(ms, rc_per_rank, world, device="cuda")

    # roofline of the cycle kernel: algorithmic bytes / its event-timed duration
    kt = [s.kernel_time(False) for s in sims]
    kernel_ms = sum(m for m, _ in kt)
    n_launch = sum(n for _, n in kt)
    stats = [s.stats() for s in sims]          # every step repeats these runs exactly
    # the period runs' end states: on this mesh every core is held up by its
    # miss latency, never by its period, so the five runs can coincide
    end_hashes = [s.state_hash() for s in sims]
    alg_total = args.steps * sum(algorithmic_bytes(st, TILES * cycles, sims[0].params)
                                 for st in stats)
    alg = alg_total / n_launch                 # per launch
    avg_launch_ms = kernel_ms / n_launch
    peak, peak_kind = measured_peaks()
    achieved = alg_total / (kernel_ms / 1e3) / 1e9
    traffic = measured_traffic(args.steps * len(PERIODS) * cycles / n_launch)

    # end to end through the public API: reset, run, read the counters back
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s in sims:
            s.reset()
            s.step_async(cycles)
            s.stats()
    e2e_s = time.perf_counter() - t0
    e2e_value = e2e_steps * len(PERIODS) * TILES * cycles * world / e2e_s
    from paper_1508_03235_b300.noc import CacheCfg, Stats, Traffic
    import ctypes
    h2d = len(PERIODS) * (ctypes.sizeof(CacheCfg) + ctypes.sizeof(Traffic))
    d2h = len(PERIODS) * ctypes.sizeof(Stats)

    batch = surrogate = None
    if not args.no_batch:
        batch = batch_section(args.batch_n, args.batch_cycles, args.batch_rect)
        surrogate = surrogate_section()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cycles_per_period=args.cpu_cycles)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Philox reference streams; the paper's traces are unavailable)",
            "config": workload_config({"cycles_per_run": cycles, "tiling": list(tiling),
                                       "thread_map": noc.THREAD_MAPS[sims[0].thread_map()],
                                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": "noc::run_kernel",
                         "launches": n_launch, "avg_launch_ms": avg_launch_ms,
                         "alg_bytes_per_launch": alg},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "period_runs": {"periods": list(PERIODS), "refs": [st["refs"] for st in stats],
                            "distinct_end_states": len(set(end_hashes))},
            "batch": batch,
            "surrogate": surrogate,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def replica_throughput(ms, units_per_rank, world, device="cpu"):
    """Whole-job throughput of `world` independent replicas: every rank did
    `units_per_rank` units; the job took the slowest rank's time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms = float(tm.item())
    return ms, units_per_rank * world / (ms / 1e3)


# --------------------------------------------------------------------- batch + surrogate
def batch_section(n, cycles, rect, thread_map=2):
    """The batched-engine half of the metric: n independent design points
    (mixed sizes, loads, mixes and L2 policies) in one persistent launch per
    memory wave, against the same instances run one at a time through the
    single-simulation path on the same GPU."""
    import torch

    from paper_1508_03235_b300 import noc
    pts = I.batch_design_points(n, seed=0)
    for p in pts:
        p.pop("design")
    tiles = sum(p["mesh_w"] * p["mesh_h"] for p in pts)
    b = noc.Batch(pts, cycles, rect=rect, collect_hash=False, thread_map=thread_map)
    b.run()                                   # warm-up (also checks every instance)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run()
    tb = time.perf_counter() - t0
    waves, launches = b.waves, b.launches
    b.close()
    # one at a time: each instance created (allocation untimed), run to its
    # cycle count and read back, before the next starts
    for p in pts[:2]:
        noc.Sim(p).step(100)
    torch.cuda.synchronize()
    t1 = 0.0
    for p in pts:
        s = noc.Sim(p, thread_map=thread_map)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.reset()
        s.step_async(cycles)
        s.stats()
        t1 += time.perf_counter() - t0
        s.close()
        del s
    return {"instances": n, "cycles": cycles, "rect": rect,
            "thread_map": noc.THREAD_MAPS[thread_map], "waves": waves,
            "batched_sims_per_s": n / tb, "one_at_a_time_sims_per_s": n / t1,
            "speedup": t1 / tb, "batched_router_cycles_per_s": tiles * cycles / tb,
            "one_at_a_time_router_cycles_per_s": tiles * cycles / t1,
            "workload": "design points: side U{8..128}, period U{2..40}, Dirichlet(2,2,1) "
                        "private/shared/remote, policy U{interleaved, LSPD, LSPD+migration}"}


def surrogate_section(reps=20, replays=20):
    """Design points per second of the surrogate's inference at batch 4096, in
    device time: `reps` calls captured in a CUDA graph and replayed, so the
    host's call overhead is not in the timed region.  The one-kernel fused
    network, and beside it the layer-by-layer forward pass it replaces."""
    import torch

    from paper_1508_03235_b300 import surrogate as S
    net = S.MLP(seed=0, max_batch=4096)
    xb = torch.rand(4096, S.DIMS[0], device="cuda").to(torch.bfloat16)
    y = torch.empty(4096, S.DIMS[-1], device="cuda")
    net.infer(xb, out=y)                       # packs the weights outside the graph

    def rate(fn):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                fn()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(replays):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / (reps * replays)

    sec = rate(lambda: net.infer(xb, out=y))
    sec_layered = rate(lambda: net.forward(xb))
    flops = 2 * 4096 * sum(S.DIMS[l] * S.DIMS[l + 1] for l in range(len(S.DIMS) - 1))
    return {"batch": 4096, "design_points_per_s": 4096 / sec, "tflops": flops / sec / 1e12,
            "us_per_batch": sec * 1e6, "layered_us_per_batch": sec_layered * 1e6, "timing": "CUDA graph replay (device time)",
            "kernel": "fused tcgen05 network (mlp_infer)", "network": list(S.DIMS)}


# --------------------------------------------------------------------- CPU arms
def cpu_baseline(cycles_per_period=400):
    """The oracle as it stands, single-threaded, on the first
    `cycles_per_period` cycles of each period's run."""
    from oracle import oracle
    oracle.build()
    rc = 0
    t = 0.0
    for P in PERIODS:
        o = oracle.OracleSim(I.mesh_208(P))
        t0 = time.perf_counter()
        o.step(cycles_per_period)
        t += time.perf_counter() - t0
        rc += TILES * cycles_per_period
        o.close()
    return {"value": rc / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {cycles_per_period} cycles of each of the {len(PERIODS)} period runs "
                      f"of the 208x208 workload ({rc} router-cycles, {t:.1f} s)"}


def _oracle_instance(job):
    """One oracle run (a spawn-pool worker): router-cycles and seconds."""
    params, cycles = job
    sys.path.insert(0, ROOT)
    from oracle import oracle
    o = oracle.OracleSim(params)
    t0 = time.perf_counter()
    o.step(cycles)
    dt = time.perf_counter() - t0
    o.close()
    return params["mesh_w"] * params["mesh_h"] * cycles, dt


def oracle_configs(c3_sample=64):
    """The oracle as it stands on the other workloads, on the host cores: the
    8x8 mesh in full (20,000 cycles), the 64x64 hotspot mesh (seed 1, 100,000
    cycles), and a sample of the 512-instance batch (every 8th instance,
    20,000 cycles each) one core at a time and over all cores."""
    import multiprocessing as mp
    from oracle import oracle
    oracle.build()
    out = {}
    for name, params, cycles in (("mesh8_full", I.MESH_8["params"], I.MESH_8["cycles"]),
                                 ("mesh64_hotspot_seed1", I.mesh_64(1), 100_000)):
        rc, dt = _oracle_instance((params, cycles))
        out[name] = {"router_cycles_per_s": rc / dt, "seconds": dt, "cores": 1}
    pts = I.batch_design_points(512, seed=0)[::512 // c3_sample]
    for p in pts:
        p.pop("design")
    jobs = [(p, 20_000) for p in pts]
    t0 = time.perf_counter()
    one = [_oracle_instance(j) for j in jobs[: max(1, len(jobs) // 8)]]
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_instance, sorted(jobs, key=lambda j: -j[0]["mesh_w"]), chunksize=1)
    t2 = time.perf_counter() - t0
    out["batch_sample_1core"] = {"instances": len(one), "sims_per_s": len(one) / t1,
                                 "router_cycles_per_s": sum(r for r, _ in one) / t1, "cores": 1}
    out["batch_sample_all_cores"] = {"instances": len(jobs), "sims_per_s": len(jobs) / t2,
                                     "router_cycles_per_s": sum(r for r, _ in res) / t2,
                                     "cores": cores}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    cyc = args.ref_cycles
    for _ in range(args.warmup):
        o = oracle.OracleSim(I.mesh_208(PERIODS[0]))
        o.step(max(1, cyc // 4))
        o.close()
    times = []
    for _ in range(args.steps):
        t = 0.0
        for P in PERIODS:
            o = oracle.OracleSim(I.mesh_208(P))
            t0 = time.perf_counter()
            o.step(cyc)
            t += time.perf_counter() - t0
            o.close()
        times.append(t)
    total = sum(times)
    value = args.steps * len(PERIODS) * TILES * cyc / total
    sample = (f"each step: first {cyc} cycles of each of the {len(PERIODS)} period runs of the "
              f"208x208 workload, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Philox reference streams)",
            "config": workload_config({"cycles_per_run": cyc}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cycles", type=int, default=CYCLES, help="cycles per period run")
    ap.add_argument("--cpu-cycles", type=int, default=400)
    ap.add_argument("--ref-cycles", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-cycles", type=int, default=20_000)
    ap.add_argument("--batch-rect", type=int, default=8)
    ap.add_argument("--oracle-configs", action="store_true",
                    help="time the oracle on the 8x8, 64x64 and batch workloads (host cores) and exit")
    args = ap.parse_args()
    if args.oracle_configs:
        print(json.dumps({"oracle_configs": oracle_configs()}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
