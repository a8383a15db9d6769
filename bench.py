"""Benchmark: simulated router-cycles/s on the 208x208 mesh (43,264 tiles).

One step = the paper's largest configuration swept over injection periods
{40, 20, 10, 5, 2}: for each period, reset the simulation to cycle 0 and run
50,000 cycles (persistent cooperative launches of up to a reference window's
cycles each).  Timed on the device with CUDA events on the simulator's
stream; the state touched per run (1.4 GB of L2 tags plus L1s, queues and
links) is larger than the GPU's L2.  The timed runs' end states are checked
against the oracle's stored records of the same runs, and the oracle itself
times one whole run on a host core while the GPU arm runs.

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


def algorithmic_bytes(stats, router_cycles, p):
    """The state bytes a cycle-stepped simulator of this model must touch
    (the byte model of the measurement plan), from a run's own counters:

    * per router-cycle: the four in-link and four out-link slots read and
      written (8 x 16 B) and the core / queue scalars read and written
      (2 x 24 B);
    * per reference: one L1 set read (ways x 8 B) and one 8 B way written;
    * per L1 miss: one L2 set read (ways x 8 B) and the line's way written (8 B);
    * per ejected protocol flit: one L2 set at the handler (ways x 8 B), plus
      one 4 B directory word under the LSPD policies."""
    lspd = p.get("policy", 0) != 0
    return (router_cycles * (8 * 16 + 2 * 24) + stats["refs"] * (8 * p["l1_ways"] + 8)
            + stats["l1_miss"] * (8 * p["l2_ways"] + 8)
            + stats["ejected"] * (8 * p["l2_ways"] + (4 if lspd else 0)))


def implementation_bytes(stats, router_cycles, p):
    """The bytes of this implementation's own state layout, for comparison:
    per router-cycle the 8 link slots (8 x 16 B) and the 13-word core record
    read and written (2 x 52 B); per L1 lookup or fill one L1 set of 32-bit
    way words read and written; per L2 access one L2 set read and written; per
    injected flit a 16 B queue push and pop."""
    l1set, l2set = 4 * p["l1_ways"], 4 * p["l2_ways"]
    l1_ops = stats["l1_hit"] + stats["l1_miss"] + stats["l2lat_cnt"]
    l2_ops = stats["l2_hit"] + stats["l2_miss"] + stats["wt_hit"] + stats["mem_write"] + stats["mem_req"]
    return (router_cycles * (8 * 16 + 2 * 52) + l1_ops * 2 * l1set + l2_ops * 2 * l2set
            + stats["injected"] * 2 * 16)


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


def captured_per_cycle():
    """DRAM and L2 bytes per simulated cycle of the cycle kernel, from the
    committed ncu capture of the same kernel sources; None for each when there
    is no capture or the kernel changed since it was taken."""
    import re
    out = {"dram_bytes_per_cycle": None, "lts_bytes_per_cycle": None}
    if not os.path.exists(TRAFFIC_FILE):
        return out
    text = open(TRAFFIC_FILE).read()
    sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    if not sha or sha.group(1) != kernel_sources_sha256():
        return out
    for k in out:
        m = re.search(k + r":\s*([0-9.eE+]+)", text)
        out[k] = float(m.group(1)) if m else None
    return out


def measured_traffic(cycles_per_launch):
    """DRAM bytes (read + write) per cycle-kernel launch, scaled from the
    committed capture by cycles per launch (DRAM traffic grows in proportion
    at a fixed mesh), or None."""
    per = captured_per_cycle()["dram_bytes_per_cycle"]
    return None if per is None else per * cycles_per_launch


# --------------------------------------------------------------------- parity records
GOLDEN = os.path.join(ROOT, "tests", "golden", "full_length.json")


def golden_final(period):
    """The oracle's stored end-of-run record of the 208x208 run at `period`
    (written by tests/golden/make_full_length.py), or None."""
    if not os.path.exists(GOLDEN):
        return None
    w = json.load(open(GOLDEN))["workloads"].get(f"mesh208_period{period}")
    return w["checkpoints"][-1] if w else None


def oracle_full_run(job):
    """A spawn-process worker: the oracle as it stands runs one whole period
    run of the 208x208 workload, single-threaded; returns its wall seconds and
    end state (counters, full state hash)."""
    params, cycles = job
    sys.path.insert(0, ROOT)
    from oracle import oracle
    oracle.build()
    o = oracle.OracleSim(params)
    t0 = time.perf_counter()
    o.step(cycles)
    dt = time.perf_counter() - t0
    out = dict(seconds=dt, stats=o.stats(), state_hash=str(o.state_hash()))
    o.close()
    return out


# --------------------------------------------------------------------- GPU arm
def run_gpu(args):
    # the oracle's full period-10 run starts first, in a spawned process on
    # one host core, and runs while the GPU arm does
    cpu_job = None
    rank, world, local = dist_env()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        cpu_pool = mp.get_context("spawn").Pool(1)
        cpu_job = cpu_pool.apply_async(oracle_full_run, ((I.mesh_208(args.cpu_period), args.cycles),))

    import torch
    import torch.distributed as dist

    from paper_1508_03235_b300 import noc

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
    impl_total = args.steps * sum(implementation_bytes(st, TILES * cycles, sims[0].params)
                                  for st in stats)
    alg = alg_total / n_launch                 # per launch
    avg_launch_ms = kernel_ms / n_launch
    peak, peak_kind = measured_peaks()
    achieved = alg_total / (kernel_ms / 1e3) / 1e9
    traffic = measured_traffic(args.steps * len(PERIODS) * cycles / n_launch)
    captured = captured_per_cycle()
    us_per_cycle = 1e3 * kernel_ms / (args.steps * len(PERIODS) * cycles)

    # bit-exact check of the timed runs (outside the timed region) against the
    # oracle's stored full-length records of the same five runs
    parity = {"runs_checked": 0, "runs_equal": 0}
    if cycles == CYCLES:
        for P, st, h in zip(PERIODS, stats, end_hashes):
            rec = golden_final(P)
            if rec is None:
                continue
            parity["runs_checked"] += 1
            same = all(st[k] == v for k, v in rec["stats"].items()) and str(h) == rec["state_hash"]
            parity["runs_equal"] += int(same)
        parity["against"] = "tests/golden/full_length.json (the oracle's records of the five runs)"

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

    load_sweep = None if args.no_load_sweep else load_sweep_section(tiling, sims[0].thread_map())
    phases = None if args.no_load_sweep else phase_section(tiling, sims[0].thread_map())
    batch = surrogate = None
    if not args.no_batch:
        batch = batch_section(args.batch_n, args.batch_cycles, rank=rank, world=world)
        surrogate = surrogate_section(accuracy=not args.no_surrogate_accuracy)

    cpu = None
    if cpu_job is not None:
        res = cpu_job.get()
        cpu_pool.close()
        cpu_pool.join()
        P = args.cpu_period
        rc = TILES * cycles
        gpu_st = stats[PERIODS.index(P)] if P in PERIODS else None
        cpu = {"value": rc / res["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "host_cores": os.cpu_count(),
               "sample": f"one whole run of the workload: the 208x208 mesh at period {P}, "
                         f"{cycles} cycles from cycle 0 ({rc} router-cycles, "
                         f"{res['seconds']:.1f} s, single thread, in a spawned process while "
                         f"the GPU arm ran)",
               "gpu_equal": (gpu_st is not None and all(gpu_st[k] == v for k, v in res["stats"].items())
                             and str(end_hashes[PERIODS.index(P)]) == res["state_hash"])}
        if not args.no_c3_baseline:
            cpu["batch_workload"] = oracle_batch_sample(args.c3_every, args.batch_cycles)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Philox reference streams; the paper's traces are unavailable)",
            "config": workload_config({"cycles_per_run": cycles, "tiling": list(tiling),
                                       "thread_map": noc.THREAD_MAPS[sims[0].thread_map()],
                                       "kernel_build": sims[0].variant(),
                                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": "noc::run_kernel",
                         "launches": n_launch, "avg_launch_ms": avg_launch_ms,
                         "us_per_simulated_cycle": us_per_cycle,
                         "alg_bytes_per_launch": alg,
                         "alg_bytes_per_router_cycle": alg_total / (rc_per_rank),
                         "byte_model": "128 B links + 48 B core/queue scalars per router-cycle; "
                                       "L1 set per reference; L2 set per L1 miss; L2 set per "
                                       "ejected flit (+4 B directory word under LSPD)",
                         "implementation_bytes_frac": impl_total / (kernel_ms / 1e3) / 1e9 / peak,
                         "dram_bytes_per_cycle": captured["dram_bytes_per_cycle"],
                         "lts_bytes_per_cycle": captured["lts_bytes_per_cycle"]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "parity": parity,
            "period_runs": {"periods": list(PERIODS), "refs": [st["refs"] for st in stats],
                            "distinct_end_states": len(set(end_hashes))},
            "load_sweep": load_sweep,
            "phase_profile": phases,
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


# --------------------------------------------------------------------- phase profile
def phase_section(tiling, thread_map, warm=2_000, cycles=4_000):
    """Where a warp's time goes in the plain loop (context): the 208x208
    period-10 run on the build with per-phase clock reads (noc_set_phase_profile;
    that build keeps its own registers, so its cycle is a little slower), SM
    clocks per warp and simulated cycle after a warm-up."""
    from paper_1508_03235_b300 import noc
    s = noc.Sim(I.mesh_208(10), tiling=tiling, thread_map=thread_map)
    s.step(warm)
    s.set_phase_profile(True)
    s.kernel_time(True)
    s.step(cycles)
    ms, _ = s.kernel_time(False)
    prof = s.phase_profile()
    s.close()
    return {"clocks_per_warp_cycle": {k: round(prof[k], 1) for k in noc.Sim.PHASES},
            "warp_cycles": prof["warp_cycles"], "us_per_cycle_profiled_build": 1e3 * ms / cycles,
            "cycles": f"{warm}..{warm + cycles} of the period-10 run"}


# --------------------------------------------------------------------- load dependence
# offered loads 0.0025 .. 0.04 flits per node-cycle, across the saturation of
# uniform traffic on a 208-wide mesh (about 0.016)
LOAD_PERIODS = (400, 200, 100, 50, 25)


def load_sweep_section(tiling, thread_map, warm=2_000, cycles=5_000):
    """Context for the period sweep, whose five runs are one simulation (on
    the 208x208 mesh a core waits on its misses, never on its period): the
    same mesh, tiling and thread order with network-only traffic (each core
    sends a one-flit probe to a uniform random tile every `period` cycles, for
    periods that take the offered load across the network's saturation).  Kernel time per simulated cycle,
    accepted flits per node-cycle and deflections per flit, per period."""
    from paper_1508_03235_b300 import noc
    out = []
    for P in LOAD_PERIODS:
        p = I.sim_params(208, 208, seed=I.MESH_208_SEED, traf=I.traffic(period=P, mode=I.MODE_NETWORK),
                         cache=I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1, svc_q=1024))
        s = noc.Sim(p, tiling=tiling, thread_map=thread_map)
        s.step(warm)
        a = s.stats()
        s.kernel_time(True)
        s.step(cycles)
        ms, _ = s.kernel_time(False)
        b = s.stats()
        ej = b["ejected"] - a["ejected"]
        out.append({"period": P, "us_per_cycle": 1e3 * ms / cycles,
                    "router_cycles_per_s": TILES * cycles / (ms / 1e3),
                    "offered_flits_per_node_cycle": 1.0 / P,
                    "accepted_flits_per_node_cycle": ej / (TILES * cycles),
                    "deflections_per_flit": (b["deflections"] - a["deflections"]) / max(ej, 1),
                    "in_flight": b["in_flight"]})
        s.close()
    return {"traffic": "network-only probes to uniform random tiles, one per core per period",
            "cycles": cycles, "after_warmup_cycles": warm, "runs": out}


# --------------------------------------------------------------------- batch + surrogate
def batch_section(n, cycles, rank=0, world=1, one_at_a_time_map=2):
    """The batched-engine half of the metric: n independent design points
    (mixed sizes, loads, mixes and L2 policies) in one persistent launch per
    kernel-variant group and memory wave, with the autotuner's layout for each
    group, against the same instances run one at a time through the
    single-simulation path on the same GPU.  With several ranks the instances
    are split by cost (shard.partition_by_cost), each rank runs its share, the
    job takes the slowest rank's time, and the per-instance results are
    gathered on every rank and checked for completeness."""
    import torch

    from paper_1508_03235_b300 import noc, shard
    pts = I.batch_design_points(n, seed=0)
    for p in pts:
        p.pop("design")
    parts = shard.partition_by_cost([shard.instance_cost(p, cycles) for p in pts], world)
    mine = parts[rank]
    local_pts = [pts[i] for i in mine]
    tiles = sum(p["mesh_w"] * p["mesh_h"] for p in pts)
    b = noc.Batch(local_pts, cycles, collect_hash=False)
    layouts = {}
    for k, i in enumerate(mine):
        layouts.setdefault(b.group(k), b.layouts[k])
    b.run()                                   # warm-up (also checks every instance)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run()
    tb = time.perf_counter() - t0
    waves, launches = b.waves, b.launches
    local = {i: {k: b.stats(k)[k2] for k2 in ("ejected", "deflections", "l2lat_sum")}
             for k, i in enumerate(mine)}
    b.close()
    merged = shard.gather_results(local, n, world)
    # one at a time: each instance created (allocation untimed), run to its
    # cycle count and read back, before the next starts
    for p in local_pts[:2]:
        noc.Sim(p).step(100)
    torch.cuda.synchronize()
    t1 = 0.0
    for p in local_pts:
        s = noc.Sim(p, thread_map=one_at_a_time_map)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.reset()
        s.step_async(cycles)
        s.stats()
        t1 += time.perf_counter() - t0
        s.close()
        del s
    tb = replica_throughput(tb * 1e3, 1, world, device="cuda")[0] / 1e3   # the slowest rank's
    t1 = replica_throughput(t1 * 1e3, 1, world, device="cuda")[0] / 1e3
    return {"instances": n, "cycles": cycles, "waves": waves, "ranks": world,
            "layouts": {tune_group_name(g): {"rect": lay[0], "strips": bool(lay[1]),
                                             "thread_map": noc.THREAD_MAPS[lay[2]]}
                        for g, lay in sorted(layouts.items())},
            "layout_source": "autotuner (tune.tune_batch) per kernel-variant group",
            "instances_gathered": len(merged),
            "batched_sims_per_s": n / tb, "one_at_a_time_sims_per_s": n / t1,
            "speedup": t1 / tb, "batched_router_cycles_per_s": tiles * cycles / tb,
            "one_at_a_time_router_cycles_per_s": tiles * cycles / t1,
            "workload": "design points: side U{8..128}, period U{2..40}, Dirichlet(2,2,1) "
                        "private/shared/remote, policy U{interleaved, LSPD, LSPD+migration}"}


def tune_group_name(g):
    from paper_1508_03235_b300 import tune
    return tune.GROUP_NAMES[g]


def surrogate_section(reps=20, replays=20, accuracy=True):
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
    out = {"batch": 4096, "design_points_per_s": 4096 / sec, "tflops": flops / sec / 1e12,
           "us_per_batch": sec * 1e6, "layered_us_per_batch": sec_layered * 1e6,
           "timing": "CUDA graph replay (device time)",
           "kernel": "fused tcgen05 network (mlp_infer)", "network": list(S.DIMS)}
    # a pool screened four batches at a time: one CTA per 128 design points,
    # so 128 SMs work instead of 32
    pool = S.MLP(seed=0, max_batch=16384)
    xp = torch.rand(16384, S.DIMS[0], device="cuda").to(torch.bfloat16)
    yp = torch.empty(16384, S.DIMS[-1], device="cuda")
    pool.infer(xp, out=yp)
    sec_pool = rate(lambda: pool.infer(xp, out=yp))
    out["pool_batch_16384"] = {"design_points_per_s": 16384 / sec_pool, "us_per_batch": sec_pool * 1e6}
    if accuracy:
        # held-out accuracy against the exact simulator: 2,000 training and
        # 500 held-out design points of the batch workload, 20,000 cycles each
        ev = S.evaluate(train=2_000, holdout=500, cycles=20_000, seeds=(0,))
        run = ev["runs"][0]
        sim_rate = (ev["train"] + ev["holdout"]) / ev["simulate_s"]
        out.update(held_out_mre=run["mre"], held_out_points=ev["holdout"],
                   train_points=ev["train"], screen_recall_top1pct=run["screen_recall"],
                   screen_random_recall=run["random_recall"],
                   simulator_design_points_per_s=sim_rate,
                   speedup_vs_simulator=(4096 / sec) / sim_rate)
    return out


# --------------------------------------------------------------------- CPU arms
def oracle_batch_sample(every=32, cycles=20_000):
    """The oracle as it stands on a sample of the batch workload (every
    `every`-th of the 512 design points, `cycles` cycles each), one process
    per host core: simulations per second over all cores (wall time) and on
    one core (the processes' summed times)."""
    import multiprocessing as mp
    pts = I.batch_design_points(512, seed=0)[::every]
    for p in pts:
        p.pop("design")
    jobs = sorted([(p, cycles) for p in pts], key=lambda j: -j[0]["mesh_w"])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, len(jobs))) as pool:
        res = pool.map(_oracle_instance, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    busy = sum(dt for _, dt in res)
    rc = sum(r for r, _ in res)
    return {"instances": len(jobs), "cycles": cycles, "cores": min(cores, len(jobs)),
            "all_cores_sims_per_s": len(jobs) / wall, "all_cores_router_cycles_per_s": rc / wall,
            "one_core_sims_per_s": len(jobs) / busy, "one_core_router_cycles_per_s": rc / busy,
            "sample": f"every {every}th of the 512 design points of the batch workload"}


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
    ap.add_argument("--cpu-period", type=int, default=10,
                    help="period of the 208x208 run the oracle times (one whole run)")
    ap.add_argument("--ref-cycles", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c3-baseline", action="store_true",
                    help="skip the oracle's sample of the batch workload over the host cores")
    ap.add_argument("--c3-every", type=int, default=32)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-load-sweep", action="store_true")
    ap.add_argument("--no-surrogate-accuracy", action="store_true",
                    help="skip the surrogate's held-out accuracy (2,500 simulated design points)")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-cycles", type=int, default=20_000)
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
