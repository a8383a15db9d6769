"""Build libnoc.so (the CUDA path) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnoc.so")
SOURCES = ["noc_run00.cu", "noc_run10.cu", "noc_run01.cu", "noc_run11.cu", "noc_batch.cu",
           "noc_kernel.cu", "noc_api.cu", "noc_static.cu"]
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
    for src in sources():           # one nvcc per translation unit, in parallel
        obj = os.path.join(BUILD, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc, *flags, "-c", src, "-o", obj]))
    if any(p.wait() != 0 for p in procs):
        raise subprocess.CalledProcessError(1, "nvcc")
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
