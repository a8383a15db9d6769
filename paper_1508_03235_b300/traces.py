"""Trace-driven input: per-core address traces read from a file.

The paper drives its simulator with per-core memory-reference traces.  Here a
trace file gives each core's references in program order; the simulator's
trace mode issues core c's k-th reference at cycle k * period (or as soon as
the core is free after that), exactly like the synthetic reference stream.

Text format, one reference per line (blank lines and '#' comments ignored):

    <core> <R|W> <byte address>          # address decimal or 0x-hexadecimal

A reference becomes the model's word  line | write << 31  with
line = address // line_bytes (64-byte lines).  Binary format: a .npz archive
with one uint32 array per core named "core<c>" holding those words already.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I

WRITE_BIT = np.uint32(1 << 31)
MAX_LINE = (1 << 26) - 1          # the model's line numbers are below 2^26


def encode(address: int, write: bool, line_bytes: int = I.LINE_BYTES) -> int:
    line = address // line_bytes
    if line > MAX_LINE:
        raise ValueError(f"address {address:#x} is beyond the model's 2^26 lines")
    return line | ((1 << 31) if write else 0)


def read_text(path: str, n_cores: int, line_bytes: int = I.LINE_BYTES):
    """Per-core arrays of encoded references from a text trace."""
    per = [[] for _ in range(n_cores)]
    with open(path) as f:
        for no, raw in enumerate(f, 1):
            s = raw.split("#", 1)[0].strip()
            if not s:
                continue
            parts = s.split()
            if len(parts) != 3:
                raise ValueError(f"{path}:{no}: expected '<core> <R|W> <address>'")
            core, op, addr = int(parts[0]), parts[1].upper(), int(parts[2], 0)
            if not 0 <= core < n_cores:
                raise ValueError(f"{path}:{no}: core {core} outside 0..{n_cores - 1}")
            if op not in ("R", "W"):
                raise ValueError(f"{path}:{no}: operation must be R or W")
            if addr < 0:
                raise ValueError(f"{path}:{no}: negative address")
            per[core].append(encode(addr, op == "W", line_bytes))
    return [np.asarray(p, dtype=np.uint32) for p in per]


def write_text(path: str, traces, line_bytes: int = I.LINE_BYTES):
    """Write per-core encoded references as a text trace (interleaved by index)."""
    n = max((len(t) for t in traces), default=0)
    with open(path, "w") as f:
        f.write("# core op address\n")
        for k in range(n):
            for c, t in enumerate(traces):
                if k < len(t):
                    w = int(t[k])
                    f.write(f"{c} {'W' if w >> 31 else 'R'} {(w & MAX_LINE) * line_bytes:#x}\n")


def read_npz(path: str, n_cores: int):
    z = np.load(path)
    out = []
    for c in range(n_cores):
        a = z[f"core{c}"] if f"core{c}" in z.files else np.zeros(0, dtype=np.uint32)
        a = np.ascontiguousarray(a, dtype=np.uint32)
        if len(a) and ((a & ~WRITE_BIT) > MAX_LINE).any():
            raise ValueError(f"{path}: core {c}: line numbers must be below 2^26")
        out.append(a)
    extra = [k for k in z.files if not (k.startswith("core") and k[4:].isdigit()
                                        and int(k[4:]) < n_cores)]
    if extra:
        raise ValueError(f"{path}: unexpected arrays {extra[:4]}")
    return out


def write_npz(path: str, traces):
    np.savez(path, **{f"core{c}": np.asarray(t, dtype=np.uint32) for c, t in enumerate(traces)})


def load(path: str, n_cores: int, line_bytes: int = I.LINE_BYTES):
    return read_npz(path, n_cores) if path.endswith(".npz") else read_text(path, n_cores, line_bytes)


def trace_params(w: int, h: int, traces, period: int = 1, policy: int = I.POLICY_INTERLEAVED,
                 cache=None, seed: int = 1):
    """Simulation parameters for trace mode: the address space is sized to
    cover the largest line any trace names."""
    top = max((int((t & ~WRITE_BIT).max()) for t in traces if len(t)), default=0)
    traf = I.traffic(period=period, mode=I.MODE_TRACE)
    traf.update(priv_lines=0, shared_lines=0, remote_lines=top + 1, priv_q16=0, shared_q16=0)
    return I.sim_params(w, h, policy=policy, cache=cache, traf=traf, seed=seed)


def apply(sim, traces):
    """Hand every core its trace (a noc.Sim, or anything with set_trace)."""
    for c, t in enumerate(traces):
        if len(t):
            sim.set_trace(c, t)
