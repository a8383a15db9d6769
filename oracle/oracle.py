"""ctypes binding of the serial oracle (oracle/noc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
bench's CPU-baseline / reference leg, never by the product path.  It imports
nothing from the CUDA path; parameters come as plain dicts built by
paper_1508_03235_b300.inputs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "noc_oracle.c")
LIB = os.path.join(HERE, "liboracle_noc.so")

STAT_NAMES = (
    "injected", "ejected", "deflections", "lat_sum", "lat_max", "refs",
    "l1_hit", "l1_miss", "l2_hit", "l2_miss", "req_made", "req_rcvd",
    "reply_sent", "reply_rcvd", "dir_search", "mem_req", "mem_write", "mem_wb",
    "wt_sent", "wt_hit", "trap", "redir", "migrations", "l2lat_sum",
    "l2lat_cnt", "cq_stall", "mm_stall", "mig_sent",
)
NSTAT = len(STAT_NAMES)
HIST_BINS = 1025

FLIT_TYPES = dict(NONE=0, REQ=1, DATA=2, WT=3, DA=4, DRPOS=5, DRNEG=6, NACK=7,
                  DINV=8, MIG=9, DIRUPD=10, INV=11, PROBE=12)


class _Params(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "mesh_w", "mesh_h", "policy", "l1_sets", "l1_ways", "l2_sets", "l2_ways",
        "l1_miss_cycles", "mem_latency", "mig_window", "mig_threshold",
        "core_q", "svc_q", "mem_q", "fwd_entries", "mode", "period")] + [
        (n, C.c_uint32) for n in ("write_q16", "priv_q16", "shared_q16", "hot_q16")] + [
        ("hot_side", C.c_int32)] + [
        (n, C.c_uint32) for n in ("priv_lines", "shared_lines", "remote_lines")] + [
        ("seed", C.c_uint64), ("stream", C.c_uint32),
        ("packet_mode", C.c_int32), ("rob_entries", C.c_int32),
        ("dir_central", C.c_int32), ("dir_tile", C.c_int32), ("l1_write_back", C.c_int32),
        ("age_mode", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, -O2) into oracle/liboracle_noc.so."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i32, i64, u32, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_uint64
        P64, P32 = C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)
        L.orc_create.argtypes = [C.POINTER(_Params), C.POINTER(vp)]
        L.orc_destroy.argtypes = [vp]
        L.orc_destroy.restype = None
        L.orc_step.argtypes = [vp, i64, P64]
        L.orc_drain.argtypes = [vp, i64, C.POINTER(i64)]
        L.orc_cycle.argtypes = [vp]
        L.orc_cycle.restype = i64
        L.orc_error.argtypes = [vp, C.POINTER(i64)]
        L.orc_stats.argtypes = [vp, i32, P64]
        L.orc_hist.argtypes = [vp, i32, P64]
        L.orc_dyn_hash.argtypes = [vp]
        L.orc_dyn_hash.restype = u64
        L.orc_state_hash.argtypes = [vp]
        L.orc_state_hash.restype = u64
        L.orc_set_trace.argtypes = [vp, i32, i64, P32]
        L.orc_debug_enqueue.argtypes = [vp, i32, i32, P32]
        L.orc_debug_link.argtypes = [vp, i32, i32, P32]
        L.orc_get_links.argtypes = [vp, P32]
        L.orc_get_cache.argtypes = [vp, i32, i32, P32]
        L.orc_dir_get.argtypes = [vp, u32]
        L.orc_dir_get.restype = u32
        L.orc_get_core.argtypes = [vp, i32, P32]
        L.orc_draw_ref.argtypes = [vp, i32, u32, P32, C.POINTER(i32)]
        L.orc_philox4x64_10.argtypes = [P64, P64, P64]
        L.orc_philox4x64_10.restype = None
        L.orc_mix64.argtypes = [u64]
        L.orc_mix64.restype = u64
        _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def philox4x64_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p64(c), _p64(k), _p64(out))
    return out


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


class OracleError(RuntimeError):
    def __init__(self, code, cycle):
        super().__init__(f"oracle error {code} at cycle {cycle}")
        self.code = code
        self.cycle = cycle


class OracleSim:
    """One serial simulation. `params` is a dict from inputs.sim_params()."""

    def __init__(self, params: dict):
        self.params = dict(params)
        pr = _Params()
        for name, _ in _Params._fields_:
            setattr(pr, name, int(params.get(name, 0)))
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(pr), C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create failed with status {rc}")
        self._h = h
        self.N = params["mesh_w"] * params["mesh_h"]

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- running -----------------------------------------------------------
    def step(self, n: int, trace: bool = False, check: bool = True):
        buf = np.zeros(max(n, 1), dtype=np.uint64) if trace else None
        rc = lib().orc_step(self._h, n, _p64(buf) if trace else None)
        if rc and check:
            raise OracleError(*self.error())
        return buf[:n] if trace else rc

    def drain(self, max_cycles: int) -> int:
        taken = C.c_int64()
        rc = lib().orc_drain(self._h, max_cycles, C.byref(taken))
        if rc:
            raise OracleError(rc, self.error()[1])
        return taken.value

    @property
    def cycle(self) -> int:
        return lib().orc_cycle(self._h)

    def error(self):
        cyc = C.c_int64()
        code = lib().orc_error(self._h, C.byref(cyc))
        return code, cyc.value

    # --- results -----------------------------------------------------------
    def stats(self, tile: int = -1) -> dict:
        out = np.zeros(NSTAT, dtype=np.uint64)
        lib().orc_stats(self._h, tile, _p64(out))
        d = {n: int(v) for n, v in zip(STAT_NAMES, out)}
        d["cycle"] = self.cycle
        d["in_flight"] = d["injected"] - d["ejected"]
        return d

    def hist(self, which: int) -> np.ndarray:
        out = np.zeros(HIST_BINS, dtype=np.uint64)
        lib().orc_hist(self._h, which, _p64(out))
        return out

    def dyn_hash(self) -> int:
        return int(lib().orc_dyn_hash(self._h))

    def state_hash(self) -> int:
        return int(lib().orc_state_hash(self._h))

    # --- scripted inputs and introspection (tests) --------------------------
    def set_trace(self, core: int, refs):
        a = np.ascontiguousarray(refs, dtype=np.uint32)
        rc = lib().orc_set_trace(self._h, core, len(a), _p32(a))
        if rc:
            raise ValueError(f"orc_set_trace status {rc}")

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
        rc = lib().orc_debug_enqueue(self._h, tile, queue, _p32(a))
        if rc:
            raise ValueError(f"orc_debug_enqueue status {rc}")

    def debug_link(self, tile: int, direction: int, flit):
        a = self._flit(flit)
        rc = lib().orc_debug_link(self._h, tile, direction, _p32(a))
        if rc:
            raise ValueError(f"orc_debug_link status {rc}")

    def links(self) -> np.ndarray:
        out = np.zeros(self.N * 4 * 8, dtype=np.uint32)
        lib().orc_get_links(self._h, _p32(out))
        return out.reshape(self.N, 4, 8)

    def cache(self, tile: int, which: int) -> np.ndarray:
        p = self.params
        sets, ways = (p["l1_sets"], p["l1_ways"]) if which == 1 else (p["l2_sets"], p["l2_ways"])
        out = np.zeros(sets * ways * 4, dtype=np.uint32)
        rc = lib().orc_get_cache(self._h, tile, which, _p32(out))
        if rc:
            raise ValueError(rc)
        return out.reshape(sets, ways, 4)

    def dir_get(self, line: int) -> int:
        return int(lib().orc_dir_get(self._h, line))

    CORE_FIELDS = ("next_ref", "fsm", "fsm_line", "fsm_write", "fsm_timer", "fsm_start",
                   "om_kind", "om_line", "om_write", "om_start", "om_timer", "om_epoch",
                   "epoch", "cq_len", "sq_len", "mq_len", "fwd_n")

    def core(self, tile: int) -> dict:
        out = np.zeros(17, dtype=np.uint32)
        lib().orc_get_core(self._h, tile, _p32(out))
        return dict(zip(self.CORE_FIELDS, (int(v) for v in out)))

    def draw_ref(self, core: int, k: int):
        line = C.c_uint32()
        w = C.c_int()
        lib().orc_draw_ref(self._h, core, k, C.byref(line), C.byref(w))
        return line.value, bool(w.value)
