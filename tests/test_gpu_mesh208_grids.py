"""The 208x208 workload (period 10) under every grid the autotuner chooses
among -- the 104x3 strips cut 2x70 ... 2x74 (some strips two rows high where
the cut falls unevenly) -- and under the next-ranked shapes and other thread
orders: each run's first 2,000 cycles end in the oracle's stored record
(tests/golden/full_length.json, written by tests/golden/make_full_length.py,
which calls only the oracle): every counter, both latency histograms, the
dynamic hash and the full state hash.  Results never depend on the grid."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_length.json")
GRIDS = [((2, g), 1) for g in (70, 71, 72, 73, 74)] + [
    ((4, 35), 1), ((6, 24), 1), ((13, 11), 1), ((2, 74), 0), ((2, 70), 2), ((11, 13), 2)]


@pytest.fixture(scope="module")
def record():
    with open(GOLDEN) as fh:
        w = json.load(fh)["workloads"]["mesh208_period10"]
    return w["params"], [c for c in w["checkpoints"] if c["cycle"] == 2000][0]


@pytest.fixture(scope="module")
def sim(record):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc
    s = noc.Sim(record[0])
    yield s
    s.close()


def hist_array(d):
    a = np.zeros(1025, dtype=np.uint64)
    for k, v in d.items():
        a[int(k)] = v
    return a


@pytest.mark.parametrize("grid,thread_map", GRIDS)
def test_grid_matches_oracle_record(sim, record, grid, thread_map):
    _, rec = record
    sim.set_tiling(*grid)
    sim.set_thread_map(thread_map)
    sim.reset()
    sim.step(2000)
    assert sim.tiling() == grid and sim.variant()["loop"] == "plain"
    st = sim.stats()
    for k, v in rec["stats"].items():
        assert st[k] == v, (grid, thread_map, k, st[k], v)
    for w in (0, 1):
        assert (sim.hist(w) == hist_array(rec["hist"][w])).all(), (grid, thread_map, "histogram", w)
    assert sim.dyn_hash() == int(rec["dyn_hash"]), (grid, thread_map)
    assert sim.state_hash() == int(rec["state_hash"]), (grid, thread_map)
