"""The batch engine on the full 512-instance workload (sides 8..128, periods
2..40, Dirichlet(2,2,1) address mixes, all three L2 policies, seeds 1..512,
20,000 cycles each) in the launch configuration the bench times (the
autotuner's layout for each kernel-variant group): every instance satisfies
the model's conservation laws, and every one of the 512 equals the oracle's
record of the same run (tests/golden/batch_c3.json, written by
tests/golden/make_batch_c3.py) in all counters, the full state hash and both
latency histograms.  A stratified sample (each policy at its smallest and a
mid-size mesh, plus a 128x128 mesh) is also re-run through the oracle here,
with full histograms."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu

CYCLES = 20_000
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_c3.json")


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


@pytest.fixture(scope="module")
def c3_points():
    pts = I.batch_design_points(512, seed=0)
    for p in pts:
        p.pop("design")
    return pts


@pytest.fixture(scope="module")
def c3_batch(noc, c3_points):
    b = noc.Batch(c3_points, CYCLES)          # the tuned layouts, as the bench runs it
    b.run()
    res = [(b.stats(i), b.state_hash(i), b.hist(i, 0), b.hist(i, 1)) for i in range(len(c3_points))]
    b.close()
    return res


def sample(pts):
    pick = set()
    for pol in (0, 1, 2):
        idx = [i for i, p in enumerate(pts) if p["policy"] == pol]
        idx.sort(key=lambda i: pts[i]["mesh_w"])
        pick.add(idx[0])
        pick.add(min(idx, key=lambda i: abs(pts[i]["mesh_w"] - 64)))
    pick.add(next(i for i, p in enumerate(pts) if p["mesh_w"] == 128))
    return sorted(pick)


def compare(i, got, want):
    (gs, gh, g0, g1), (os_, oh, o0, o1) = got, want
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (i, k, gs[k], v)
    assert gh == oh, i
    assert (g0 == o0).all() and (g1 == o1).all(), i


def test_c3_invariants_every_instance(c3_points, c3_batch):
    for i, (p, (st, h, h0, h1)) in enumerate(zip(c3_points, c3_batch)):
        n = p["mesh_w"] * p["mesh_h"]
        assert st["cycle"] == CYCLES, i
        assert st["injected"] == st["ejected"] + st["in_flight"], i
        assert int(h0.sum()) == st["ejected"], i                 # one latency sample per flit
        assert int(h1.sum()) == st["l2lat_cnt"], i
        assert st["l1_hit"] + st["l1_miss"] >= st["refs"], i      # every reference looks up the L1
        assert st["ejected"] <= n * CYCLES, i                    # one ejection per tile-cycle
        assert st["lat_max"] < CYCLES, i


def test_c3_sample_matches_oracle(c3_points, c3_batch):
    from tests.oracle_pool import run_many
    idx = sample(c3_points)
    assert {c3_points[i]["policy"] for i in idx} == {0, 1, 2}
    want = run_many([c3_points[i] for i in idx], CYCLES)
    for i, w in zip(idx, want):
        compare(i, c3_batch[i], w)


def hist_digest(h) -> str:
    return hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest()[:16]


def test_c3_every_instance_matches_oracle_records(c3_points, c3_batch):
    with open(GOLDEN) as fh:
        doc = json.load(fh)
    assert doc["instances"] == len(c3_points) and doc["cycles"] == CYCLES
    bad = []
    for i, (rec, (gs, gh, g0, g1)) in enumerate(zip(doc["records"], c3_batch)):
        ok = (all(gs[k] == v for k, v in rec["stats"].items()) and str(gh) == rec["state_hash"]
              and [hist_digest(g0), hist_digest(g1)] == rec["hist_sha"])
        if not ok:
            bad.append(i)
    assert not bad, f"{len(bad)} of {len(c3_points)} instances differ: {bad[:10]}"
