"""ctypes binding of libnoc.so (the CUDA path); argument marshalling only.

Every simulated cycle runs in the library's sm_103a kernels.  PyTorch provides
the device arena (a uint8 tensor bound with noc_bind_memory) and the stream.
There is no CPU fallback: importing this module raises if the library or a
CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnoc.so")

NOC_OK = 0
THREAD_MAPS = ("perimeter first", "rows", "columns")
KERNEL_KINDS = ("general", "base", "interleaved", "lspd-local", "lspd-migrate")
ERR_NAMES = {1: "NOC_ERR_ARG", 2: "NOC_ERR_OOM", 3: "NOC_ERR_QUEUE_OVERFLOW", 4: "NOC_ERR_TIMEOUT",
             5: "NOC_ERR_CUDA", 6: "NOC_ERR_PROTOCOL", 7: "NOC_ERR_STATE", 8: "NOC_ERR_RANGE",
             9: "NOC_ERR_OWNER"}
HIST_BINS = 1025
FLIT_TYPES = dict(NONE=0, REQ=1, DATA=2, WT=3, DA=4, DRPOS=5, DRNEG=6, NACK=7, DINV=8, MIG=9,
                  DIRUPD=10, INV=11, PROBE=12)


class CacheCfg(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "l1_sets", "l1_ways", "l2_sets", "l2_ways", "l1_miss_cycles", "mem_latency",
        "mig_window", "mig_threshold", "core_q", "svc_q", "mem_q", "fwd_entries",
        "packet_mode", "rob_entries", "dir_central", "dir_tile", "l1_write_back", "age_mode")]


class Traffic(C.Structure):
    _fields_ = [("mode", C.c_int32), ("period", C.c_int32), ("write_q16", C.c_uint32),
                ("priv_q16", C.c_uint32), ("shared_q16", C.c_uint32), ("hot_q16", C.c_uint32),
                ("hot_side", C.c_int32), ("priv_lines", C.c_uint32), ("shared_lines", C.c_uint32),
                ("remote_lines", C.c_uint32), ("stream", C.c_uint32)]


STATS_FIELDS = ("cycle", "injected", "ejected", "in_flight", "deflections", "lat_sum", "lat_max",
                "refs", "l1_hit", "l1_miss", "l2_hit", "l2_miss", "req_made", "req_rcvd",
                "reply_sent", "reply_rcvd", "dir_search", "mem_req", "mem_write", "mem_wb",
                "wt_sent", "wt_hit", "trap", "redir", "migrations", "l2lat_sum", "l2lat_cnt",
                "cq_stall", "mm_stall", "mig_sent")


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in STATS_FIELDS]


class NocError(RuntimeError):
    def __init__(self, code, msg, cycle=-1):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code
        self.cycle = cycle


_lib = None


def lib():
    """Load libnoc.so; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python paper_1508_03235_b300/build.py`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32, P64, P32 = (C.c_void_p, C.c_int, C.c_int64, C.c_uint32,
                                       C.POINTER(C.c_uint64), C.POINTER(C.c_uint32))
        sig = {
            "noc_create": (i32, [i32, i32, C.POINTER(CacheCfg), i32, C.POINTER(Traffic), C.c_uint64,
                                 C.POINTER(vp)]),
            "noc_destroy": (None, [vp]),
            "noc_required_bytes": (C.c_size_t, [vp]),
            "noc_bind_memory": (i32, [vp, vp, C.c_size_t]),
            "noc_set_stream": (i32, [vp, vp]),
            "noc_reset": (i32, [vp]),
            "noc_step": (i32, [vp, i64]),
            "noc_drain": (i32, [vp, i64, C.POINTER(i64)]),
            "noc_sync": (i32, [vp, C.POINTER(i64)]),
            "noc_stats": (i32, [vp, i32, C.POINTER(Stats)]),
            "noc_latency_hist": (i32, [vp, i32, P64, i32]),
            "noc_dyn_hash": (i32, [vp, P64]),
            "noc_state_hash": (i32, [vp, P64]),
            "noc_set_hash_trace": (i32, [vp, i32]),
            "noc_hash_trace": (i32, [vp, P64, i64]),
            "noc_set_tiling": (i32, [vp, i32, i32]),
            "noc_get_tiling": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
            "noc_set_thread_map": (i32, [vp, i32]),
            "noc_set_tiles_per_thread": (i32, [vp, i32]),
            "noc_get_tiles_per_thread": (i32, [vp]),
            "noc_get_thread_map": (i32, [vp]),
            "noc_set_trace": (i32, [vp, i32, i64, P32]),
            "noc_debug_enqueue": (i32, [vp, i32, i32, P32]),
            "noc_debug_link": (i32, [vp, i32, i32, P32]),
            "noc_get_links": (i32, [vp, P32]),
            "noc_get_cache": (i32, [vp, i32, i32, P32]),
            "noc_dir_get": (i32, [vp, u32, P32]),
            "noc_get_core": (i32, [vp, i32, P32]),
            "noc_debug_wait_limit": (i32, [vp, i64, i32]),
            "noc_kernel_launches": (i64, [vp]),
            "noc_kernel_time": (i32, [vp, i32, C.POINTER(C.c_double), C.POINTER(i64)]),
            "noc_last_variant": (i32, [vp] + [C.POINTER(i32)] * 4),
            "noc_last_launch_bound": (i32, [vp]),
            "noc_set_phase_profile": (i32, [vp, i32]),
            "noc_set_checks": (i32, [vp, i32]),
            "noc_phase_profile": (i32, [vp, P64]),
            "noc_checkpoint_bytes": (C.c_size_t, [vp]),
            "noc_save": (i32, [vp, vp, C.c_size_t]),
            "noc_load": (i32, [vp, vp, C.c_size_t]),
            "noc_run_static": (i32, [i32, i32, C.POINTER(CacheCfg), i32, C.POINTER(Traffic),
                                     C.c_uint64, i64, vp, vp]),
            "noc_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, cycle=-1):
    if rc != NOC_OK:
        raise NocError(rc, lib().noc_last_error().decode(), cycle)


def _p64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def cache_struct(p: dict) -> CacheCfg:
    c = CacheCfg()
    for n, _ in CacheCfg._fields_:
        setattr(c, n, int(p.get(n, 0)))
    return c


def traffic_struct(p: dict) -> Traffic:
    t = Traffic()
    for n, _ in Traffic._fields_:
        setattr(t, n, int(p.get(n, 0)))
    return t


class Sim:
    """One simulation on the current CUDA device.  `params` is a flat dict from
    paper_1508_03235_b300.inputs.sim_params()."""

    def __init__(self, params: dict, stream=None, tiling=None, thread_map=None, tiles_per_thread=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the simulator needs a CUDA device")
        self.params = dict(params)
        self.N = params["mesh_w"] * params["mesh_h"]
        h = C.c_void_p()
        rc = lib().noc_create(params["mesh_w"], params["mesh_h"], C.byref(cache_struct(params)),
                              params.get("policy", 0), C.byref(traffic_struct(params)),
                              params.get("seed", 1), C.byref(h))
        _check(rc)
        self._h = h
        nbytes = lib().noc_required_bytes(h)
        self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = self._mem.data_ptr()
        ptr += (-ptr) % 256
        _check(lib().noc_bind_memory(h, C.c_void_p(ptr), nbytes))
        st = stream if stream is not None else torch.cuda.current_stream()
        self._stream = st
        _check(lib().noc_set_stream(h, C.c_void_p(st.cuda_stream)))
        if tiling is not None:
            self.set_tiling(*tiling)
        if thread_map is not None:
            self.set_thread_map(thread_map)
        if tiles_per_thread is not None:
            self.set_tiles_per_thread(tiles_per_thread)
        _check(lib().noc_reset(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().noc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- running -----------------------------------------------------------
    def reset(self):
        _check(lib().noc_reset(self._h))

    def step(self, n: int, trace: bool = False, sync: bool = True):
        if trace:
            _check(lib().noc_set_hash_trace(self._h, 1))
        try:
            _check(lib().noc_step(self._h, n))
            if trace or sync:
                self.sync()
            if trace:
                buf = np.zeros(max(n, 1), dtype=np.uint64)
                _check(lib().noc_hash_trace(self._h, _p64(buf), n))
                return buf[:n]
        finally:
            if trace:
                lib().noc_set_hash_trace(self._h, 0)
        return None

    def step_async(self, n: int):
        _check(lib().noc_step(self._h, n))

    def sync(self):
        cyc = C.c_int64()
        rc = lib().noc_sync(self._h, C.byref(cyc))
        _check(rc, cyc.value)

    def error(self):
        cyc = C.c_int64()
        rc = lib().noc_sync(self._h, C.byref(cyc))
        return rc, cyc.value

    def drain(self, max_cycles: int) -> int:
        taken = C.c_int64()
        _check(lib().noc_drain(self._h, max_cycles, C.byref(taken)))
        return taken.value

    def set_tiling(self, gx: int, gy: int):
        _check(lib().noc_set_tiling(self._h, gx, gy))

    def tiling(self):
        gx, gy = C.c_int(), C.c_int()
        _check(lib().noc_get_tiling(self._h, C.byref(gx), C.byref(gy)))
        return gx.value, gy.value

    def set_tiles_per_thread(self, k: int):
        """1: one tile per thread (the fast loop), 2: two (meshes beyond one
        co-resident launch), 0: automatic."""
        _check(lib().noc_set_tiles_per_thread(self._h, k))

    def tiles_per_thread(self) -> int:
        return lib().noc_get_tiles_per_thread(self._h)

    def set_thread_map(self, m: int):
        """Tile-to-thread order inside each CTA rectangle: THREAD_MAPS[m]."""
        _check(lib().noc_set_thread_map(self._h, m))

    def thread_map(self) -> int:
        return lib().noc_get_thread_map(self._h)

    def wait_limit(self, ns: int, silent_cta: int = -1):
        _check(lib().noc_debug_wait_limit(self._h, ns, silent_cta))

    @property
    def launches(self) -> int:
        return lib().noc_kernel_launches(self._h)

    def variant(self) -> dict:
        """The cycle-kernel build of the last launch: loop ("plain" or
        "traced"), kind (KERNEL_KINDS) and its way bounds (l1, l2)."""
        v = [C.c_int() for _ in range(4)]
        _check(lib().noc_last_variant(self._h, *[C.byref(x) for x in v]))
        return dict(loop=("plain", "traced", "plain, two tiles per thread")[v[0].value],
                    kind=KERNEL_KINDS[v[1].value], bounds=(v[2].value, v[3].value))

    PHASES = ("wait", "route", "publish", "phase3", "phase1")

    def set_checks(self, enable: bool = True):
        """Run later plain launches on the checked build (noc_set_checks): a
        directory entry touched away from its line's directory tile ends the
        step with NOC_ERR_OWNER."""
        _check(lib().noc_set_checks(self._h, 1 if enable else 0))

    def set_phase_profile(self, enable: bool = True):
        """Run later plain launches on the build with per-phase clock reads."""
        _check(lib().noc_set_phase_profile(self._h, 1 if enable else 0))

    def phase_profile(self) -> dict:
        """SM clocks per warp-cycle in each phase since the last call (and
        the number of warp-cycles), then cleared."""
        v = np.zeros(6, dtype=np.uint64)
        _check(lib().noc_phase_profile(self._h, _p64(v)))
        n = int(v[5])
        out = {name: (int(v[k]) / n if n else 0.0) for k, name in enumerate(self.PHASES)}
        out["warp_cycles"] = n
        return out

    def launch_bound(self) -> int:
        """Most threads per CTA of the last launch's build (320, 384 or 448
        for the plain loop)."""
        return lib().noc_last_launch_bound(self._h)

    def kernel_time(self, enable: bool = True):
        """(ms, launches) of the cycle-kernel launches recorded since the last
        call (CUDA events around each launch), then keep recording iff enable."""
        ms, n = C.c_double(), C.c_int64()
        _check(lib().noc_kernel_time(self._h, int(enable), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    # --- checkpoint / resume ------------------------------------------------
    def save(self) -> np.ndarray:
        """The whole simulation state as a host image (uint8 array)."""
        n = lib().noc_checkpoint_bytes(self._h)
        buf = np.empty(n, dtype=np.uint8)
        _check(lib().noc_save(self._h, buf.ctypes.data_as(C.c_void_p), n))
        return buf

    def load(self, image: np.ndarray):
        """Restore a state saved by save() from a simulation of the same
        configuration."""
        a = np.ascontiguousarray(image, dtype=np.uint8)
        _check(lib().noc_load(self._h, a.ctypes.data_as(C.c_void_p), a.nbytes))

    # --- results -----------------------------------------------------------
    def stats(self, tile: int = -1) -> dict:
        s = Stats()
        _check(lib().noc_stats(self._h, tile, C.byref(s)))
        return {n: int(getattr(s, n)) for n in STATS_FIELDS}

    @property
    def cycle(self) -> int:
        return self.stats()["cycle"]

    def hist(self, which: int) -> np.ndarray:
        out = np.zeros(HIST_BINS, dtype=np.uint64)
        _check(lib().noc_latency_hist(self._h, which, _p64(out), HIST_BINS))
        return out

    def dyn_hash(self) -> int:
        v = np.zeros(1, dtype=np.uint64)
        _check(lib().noc_dyn_hash(self._h, _p64(v)))
        return int(v[0])

    def state_hash(self) -> int:
        v = np.zeros(1, dtype=np.uint64)
        _check(lib().noc_state_hash(self._h, _p64(v)))
        return int(v[0])

    # --- scripted inputs and introspection ---------------------------------
    def set_trace(self, core: int, refs):
        a = np.ascontiguousarray(refs, dtype=np.uint32)
        _check(lib().noc_set_trace(self._h, core, len(a), _p32(a)))

    @staticmethod
    def _flit(f):
        if isinstance(f, dict):
            f = [FLIT_TYPES[f["type"]] if isinstance(f["type"], str) else f["type"],
                 f.get("src", 0), f["dst"], f.get("inject", 0), f.get("line", 0),
                 f.get("a", 0), f.get("e", 0), f.get("age", 0)]
        a = np.zeros(8, dtype=np.uint32)
        a[:len(f)] = f          # 7 words (no age) or 8
        return a

    def debug_enqueue(self, tile: int, queue: int, flit):
        a = self._flit(flit)
        _check(lib().noc_debug_enqueue(self._h, tile, queue, _p32(a)))

    def debug_link(self, tile: int, direction: int, flit):
        a = self._flit(flit)
        _check(lib().noc_debug_link(self._h, tile, direction, _p32(a)))

    def links(self) -> np.ndarray:
        out = np.zeros(self.N * 4 * 8, dtype=np.uint32)
        _check(lib().noc_get_links(self._h, _p32(out)))
        return out.reshape(self.N, 4, 8)

    def cache(self, tile: int, which: int) -> np.ndarray:
        p = self.params
        sets, ways = (p["l1_sets"], p["l1_ways"]) if which == 1 else (p["l2_sets"], p["l2_ways"])
        out = np.zeros(sets * ways * 4, dtype=np.uint32)
        _check(lib().noc_get_cache(self._h, tile, which, _p32(out)))
        return out.reshape(sets, ways, 4)

    def dir_get(self, line: int) -> int:
        v = np.zeros(1, dtype=np.uint32)
        _check(lib().noc_dir_get(self._h, line, _p32(v)))
        return int(v[0])

    CORE_FIELDS = ("next_ref", "fsm", "fsm_line", "fsm_write", "fsm_timer", "fsm_start",
                   "om_kind", "om_line", "om_write", "om_start", "om_timer", "om_epoch",
                   "epoch", "cq_len", "sq_len", "mq_len", "fwd_n")

    def core(self, tile: int) -> dict:
        out = np.zeros(17, dtype=np.uint32)
        _check(lib().noc_get_core(self._h, tile, _p32(out)))
        return dict(zip(self.CORE_FIELDS, (int(v) for v in out)))


# --------------------------------------------------------------------------- batch
class InstanceDesc(C.Structure):
    _fields_ = [("mesh_w", C.c_int32), ("mesh_h", C.c_int32), ("l2_policy", C.c_int32),
                ("reserved", C.c_int32), ("cache", CacheCfg), ("traffic", Traffic),
                ("seed", C.c_uint64), ("cycles", C.c_int64)]


def _batch_sigs(L):
    vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
    sig = {
        "noc_batch_create": (i32, [i32, C.POINTER(InstanceDesc), C.POINTER(vp)]),
        "noc_batch_destroy": (None, [vp]),
        "noc_batch_min_bytes": (C.c_size_t, [vp]),
        "noc_batch_total_bytes": (C.c_size_t, [vp]),
        "noc_batch_bind_memory": (i32, [vp, vp, C.c_size_t]),
        "noc_batch_set_stream": (i32, [vp, vp]),
        "noc_batch_set_rect": (i32, [vp, i32]),
        "noc_batch_set_thread_map": (i32, [vp, i32]),
        "noc_batch_set_strips": (i32, [vp, i32]),
        "noc_batch_set_collect_hash": (i32, [vp, i32]),
        "noc_batch_run": (i32, [vp]),
        "noc_batch_waves": (i32, [vp]),
        "noc_batch_error": (i32, [vp, i32, C.POINTER(i64)]),
        "noc_batch_stats": (i32, [vp, i32, C.POINTER(Stats)]),
        "noc_batch_state_hash": (i32, [vp, i32, C.POINTER(C.c_uint64)]),
        "noc_batch_latency_hist": (i32, [vp, i32, i32, C.POINTER(C.c_uint64), i32]),
        "noc_batch_kernel_launches": (i64, [vp]),
        "noc_batch_variant": (i32, [vp, i32] + [C.POINTER(i32)] * 3),
        "noc_batch_group": (i32, [vp, i32]),
        "noc_batch_set_layout": (i32, [vp, i32, i32, i32, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _descs(params_list, cycles):
    n = len(params_list)
    if isinstance(cycles, int):
        cycles = [cycles] * n
    arr = (InstanceDesc * n)()
    for d, p, c in zip(arr, params_list, cycles):
        d.mesh_w, d.mesh_h, d.l2_policy = p["mesh_w"], p["mesh_h"], p.get("policy", 0)
        d.cache = cache_struct(p)
        d.traffic = traffic_struct(p)
        d.seed = p.get("seed", 1)
        d.cycles = int(c)
    return arr


def batch_groups(params_list):
    """The kernel-variant group (noc_batch_group) of each instance: host-only,
    no device memory is taken."""
    L = lib()
    _batch_sigs(L)
    h = C.c_void_p()
    _check(L.noc_batch_create(len(params_list), _descs(params_list, 1), C.byref(h)))
    try:
        return [L.noc_batch_group(h, i) for i in range(len(params_list))]
    finally:
        L.noc_batch_destroy(h)


class Batch:
    """Independent simulations run together by the batch engine.  `params_list`
    holds inputs.sim_params() dicts; `cycles` is one count or one per instance.
    The instances' state lives in a torch uint8 pool of `pool_bytes` (default:
    all instances at once, capped at 80% of free device memory); instances
    that do not fit run in later waves.  The layout knobs (rect, strips,
    thread_map) apply to every instance when given; otherwise each instance
    takes the autotuner's cached choice for its kernel-variant group
    (tuned=True) or the library default."""

    def __init__(self, params_list, cycles, stream=None, rect=None, collect_hash=True,
                 pool_bytes=None, thread_map=None, strips=None, tuned=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the batch engine needs a CUDA device")
        L = lib()
        _batch_sigs(L)
        n = len(params_list)
        h = C.c_void_p()
        _check(L.noc_batch_create(n, _descs(params_list, cycles), C.byref(h)))
        self._h = h
        self.n = n
        total = L.noc_batch_total_bytes(h)
        free, _ = torch.cuda.mem_get_info()
        want = pool_bytes if pool_bytes is not None else min(total, int(free * 0.8))
        want = max(int(want), L.noc_batch_min_bytes(h))
        self._pool = torch.empty(want + 256, dtype=torch.uint8, device="cuda")
        ptr = self._pool.data_ptr()
        ptr += (-ptr) % 256
        _check(L.noc_batch_bind_memory(h, C.c_void_p(ptr), want))
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(L.noc_batch_set_stream(h, C.c_void_p(st.cuda_stream)))
        # layout: what the caller gives, else the autotuner's choice for each
        # instance's kernel-variant group, else 8x8 squares, perimeter first
        self.layouts = []
        cache = {}
        if tuned and rect is None and strips is None and thread_map is None:
            from . import tune
            for g in range(len(tune.GROUP_NAMES)):
                cache[g] = tune.cached_batch_layout(g)
        for i in range(n):
            lay = cache.get(L.noc_batch_group(h, i)) or (8, False, 0)
            lay = (rect if rect is not None else lay[0], strips if strips is not None else lay[1],
                   thread_map if thread_map is not None else lay[2])
            self.layouts.append(lay)
            _check(L.noc_batch_set_layout(h, i, lay[0], 1 if lay[1] else 0, lay[2]))
        _check(L.noc_batch_set_collect_hash(h, 1 if collect_hash else 0))

    def close(self):
        if getattr(self, "_h", None):
            lib().noc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, check=True):
        rc = lib().noc_batch_run(self._h)
        if check:
            _check(rc)
        return rc

    @property
    def waves(self) -> int:
        return lib().noc_batch_waves(self._h)

    @property
    def launches(self) -> int:
        return lib().noc_batch_kernel_launches(self._h)

    def error(self, i):
        cyc = C.c_int64()
        rc = lib().noc_batch_error(self._h, i, C.byref(cyc))
        return rc, cyc.value

    def group(self, i) -> int:
        """Kernel-variant group of instance i (0-2 interleaved builds by way
        class, 3 base, 4 general)."""
        return lib().noc_batch_group(self._h, i)

    def set_layout(self, i, rect, strips, thread_map):
        """CTA rectangle side, strips and thread order of instance i (-1: all)."""
        _check(lib().noc_batch_set_layout(self._h, i, rect, 1 if strips else 0, thread_map))

    def variant(self, i) -> dict:
        """The batch-kernel build that runs instance i: kind and way bounds."""
        v = [C.c_int() for _ in range(3)]
        _check(lib().noc_batch_variant(self._h, i, *[C.byref(x) for x in v]))
        return dict(kind=KERNEL_KINDS[v[0].value], bounds=(v[1].value, v[2].value))

    def stats(self, i) -> dict:
        s = Stats()
        _check(lib().noc_batch_stats(self._h, i, C.byref(s)))
        return {n: int(getattr(s, n)) for n in STATS_FIELDS}

    def state_hash(self, i) -> int:
        v = C.c_uint64()
        _check(lib().noc_batch_state_hash(self._h, i, C.byref(v)))
        return int(v.value)

    def hist(self, i, which) -> np.ndarray:
        out = np.zeros(HIST_BINS, dtype=np.uint64)
        _check(lib().noc_batch_latency_hist(self._h, i, which, _p64(out), HIST_BINS))
        return out
