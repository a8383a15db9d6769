"""Build libnoc.so (the CUDA path) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnoc.so")
# (source, preprocessor defines): the cycle kernel is compiled once per variant
WAY_BOUNDS = ((4, 8), (4, 16), (16, 16))
POLICIES = (0, 1, 2)   # interleaved, LSPD local placement, LSPD migration
UNITS = ([("noc_run_variant.cu", {"NOC_HASH": h, "NOC_DRAIN": d, "NOC_W1": w1, "NOC_W2": w2})
          for (w1, w2) in WAY_BOUNDS for (h, d) in ((0, 0), (1, 0), (0, 1))]
         # the plain loop specialised to one L2 policy (0 interleaved, 1 LSPD
         # local placement, 2 LSPD migration) with the class's exact ways
         + [("noc_run_variant.cu", {"NOC_HASH": 0, "NOC_DRAIN": 0, "NOC_W1": w1, "NOC_W2": w2,
                                    "NOC_FIXED_POLICY": pol, "NOC_FIXED_MODE": 0, "NOC_EXACT_WAYS": 1})
            for (w1, w2) in WAY_BOUNDS for pol in POLICIES]
         + [("noc_run_variant.cu", {"NOC_HASH": 0, "NOC_DRAIN": 0, "NOC_W1": w1, "NOC_W2": w2,
                                    "NOC_BASE": 1}) for (w1, w2) in WAY_BOUNDS]
         # the plain loop again, for CTAs of at most 320 threads (more registers)
         + [("noc_run_variant.cu", dict(spec, NOC_HASH=0, NOC_DRAIN=0, NOC_W1=w1, NOC_W2=w2, NOC_NARROW=1))
            for (w1, w2) in WAY_BOUNDS
            for spec in [{}, {"NOC_BASE": 1}]
            + [{"NOC_FIXED_POLICY": pol, "NOC_FIXED_MODE": 0, "NOC_EXACT_WAYS": 1} for pol in POLICIES]]
         # and for CTAs of up to 448 threads (128 registers)
         + [("noc_run_variant.cu", dict(spec, NOC_HASH=0, NOC_DRAIN=0, NOC_W1=w1, NOC_W2=w2, NOC_XL=1))
            for (w1, w2) in WAY_BOUNDS
            for spec in [{}, {"NOC_BASE": 1}]
            + [{"NOC_FIXED_POLICY": pol, "NOC_FIXED_MODE": 0, "NOC_EXACT_WAYS": 1} for pol in POLICIES]]
         # the general plain loop with the single-writer checks (noc_set_checks)
         + [("noc_run_variant.cu", {"NOC_HASH": 0, "NOC_DRAIN": 0, "NOC_W1": w1, "NOC_W2": w2, "NOC_CHECKS": 1})
            for (w1, w2) in WAY_BOUNDS]
         # and with per-phase clock reads (noc_set_phase_profile)
         + [("noc_run_variant.cu", dict(spec, NOC_HASH=0, NOC_DRAIN=0, NOC_W1=w1, NOC_W2=w2,
                                        NOC_PHASE_PROFILE=1))
            for (w1, w2) in WAY_BOUNDS
            for spec in ({}, {"NOC_BASE": 1},
                         {"NOC_FIXED_POLICY": 0, "NOC_FIXED_MODE": 0, "NOC_EXACT_WAYS": 1})]
         + [("noc_batch.cu", {"NOC_W1": w1, "NOC_W2": w2}) for (w1, w2) in WAY_BOUNDS]
         + [("noc_batch.cu", {"NOC_W1": w1, "NOC_W2": w2, "NOC_BASE": 1}) for (w1, w2) in WAY_BOUNDS]
         + [("noc_batch.cu", {"NOC_W1": w1, "NOC_W2": w2, "NOC_FIXED_POLICY": pol, "NOC_FIXED_MODE": 0,
                              "NOC_EXACT_WAYS": 1}) for (w1, w2) in WAY_BOUNDS for pol in POLICIES]
         + [("noc_run_multi.cu", {"NOC_W1": w1, "NOC_W2": w2}) for (w1, w2) in WAY_BOUNDS]
         + [("noc_kernel.cu", {}), ("noc_api.cu", {}), ("noc_static.cu", {}), ("mlp.cu", {})])
SOURCES = sorted({u[0] for u in UNITS})
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES]


def deps():
    out = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out + [os.path.join(ROOT, "include", "noc.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        flags.append("-Xptxas=-v")
    objs, procs = [], []
    for k, (src, defs) in enumerate(UNITS):   # one nvcc per unit, run in parallel
        obj = os.path.join(BUILD, f"{k:02d}_{src}.{os.getpid()}.o")
        objs.append(obj)
        dflags = [f"-D{n}={v}" for n, v in defs.items()]
        procs.append(subprocess.Popen([nvcc, *flags, *dflags, "-c", os.path.join(CSRC, src),
                                       "-o", obj]))
    if any(p.wait() != 0 for p in procs):
        raise subprocess.CalledProcessError(1, "nvcc")
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
