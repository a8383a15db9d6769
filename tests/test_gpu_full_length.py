"""Bit-exact parity at the workloads' full configured lengths.

The 64x64 hotspot mesh (seeds 1-4, 100,000 cycles each) and the 208x208 mesh
(the paper's largest scale, 43,264 tiles) at every injection period of the
benchmark sweep (50,000 cycles each), run through libnoc.so in the
benchmark's launch configuration (the tuned tiling and thread order), against
the oracle's records of the same runs in tests/golden/full_length.json
(written by tests/golden/make_full_length.py, which calls only the oracle).

Each run is compared at three checkpoints (2,000 / 20,000 / 100,000 cycles
and 2,000 / 10,000 / 50,000 cycles): every counter, both latency histograms,
the dynamic hash and the full state hash (every valid L1 and L2 way, queue
entry, memory-FIFO entry and link).  A second simulation of each 208x208 run
takes all 50,000 cycles in one noc_step call, exactly as the benchmark does.
This is the paper's GPU-equals-serial validation (Sec. 7.3) at its largest
mesh, over whole runs in which L1 and L2 victims are chosen all the time."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_length.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)["workloads"]


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def hist_array(d):
    a = np.zeros(1025, dtype=np.uint64)
    for k, v in d.items():
        a[int(k)] = v
    return a


def assert_checkpoint(g, rec, name):
    gs = g.stats()
    for k, v in rec["stats"].items():
        assert gs[k] == v, (name, rec["cycle"], k, gs[k], v)
    assert gs["cycle"] == rec["cycle"]
    for w in (0, 1):
        assert (g.hist(w) == hist_array(rec["hist"][w])).all(), (name, rec["cycle"], "histogram", w)
    assert g.dyn_hash() == int(rec["dyn_hash"]), (name, rec["cycle"], "dynamic hash")
    assert g.state_hash() == int(rec["state_hash"]), (name, rec["cycle"], "full state hash")


def bench_sim(noc, params):
    from paper_1508_03235_b300 import tune
    return noc.Sim(params, tiling=tune.cached_tiling(params), thread_map=tune.cached_thread_map(params))


def run_checkpoints(noc, golden, name):
    w = golden[name]
    g = bench_sim(noc, w["params"])
    done = 0
    for rec in w["checkpoints"]:
        g.step(rec["cycle"] - done)
        done = rec["cycle"]
        assert_checkpoint(g, rec, name)
    assert g.variant()["loop"] == "plain"
    return g


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_mesh64_hotspot_full_length(noc, golden, seed):
    g = run_checkpoints(noc, golden, f"mesh64_hotspot_seed{seed}")
    assert g.variant() == dict(loop="plain", kind="interleaved", bounds=(4, 8))


@pytest.mark.parametrize("period", [40, 20, 10, 5, 2])
def test_mesh208_full_length(noc, golden, period):
    name = f"mesh208_period{period}"
    g = run_checkpoints(noc, golden, name)
    assert g.variant() == dict(loop="plain", kind="interleaved", bounds=(4, 16))
    assert g.launch_bound() == 320              # 104x3 strips: the narrow build
    # the benchmark's own sequence: reset, then the whole run in one call
    g.reset()
    last = golden[name]["checkpoints"][-1]
    g.step(last["cycle"])
    assert_checkpoint(g, last, name)
