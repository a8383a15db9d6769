"""The L1 write-back option (dirty L1 copies; a dirty victim written to the L2
that supplied it) on the CUDA path against the oracle: the hand-worked
eviction timeline, every cycle's state hash under the three policies with
drains, both cycle loops at 8x8 and 64x64, and write-back instances in a
batch."""
import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def traced(g, o, n):
    tg, to = g.step(n, trace=True), o.step(n, trace=True)
    bad = np.nonzero(tg != to)[0]
    assert len(bad) == 0, f"first per-cycle hash mismatch at cycle {o.cycle - n + bad[0]}"


def same(g, o):
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (k, gs[k], v)
    for w in (0, 1):
        assert (g.hist(w) == o.hist(w)).all()
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


def test_write_back_eviction_timeline(noc, oracle_mod):
    # core 0 reads line 8 (home tile 8), writes it as an L1 hit, then four more
    # lines of the same L1 set evict it: the write to tile 8 leaves only then
    l1_sets = I.cache_cfg()["l1_sets"]
    refs = [8, 8 | (1 << 31)] + [8 + k * l1_sets for k in range(1, 5)]
    traf = I.traffic(period=200, mode=I.MODE_TRACE)
    p = I.sim_params(3, 3, cache=I.cache_cfg(l1_write_back=1), traf=traf)
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    g.set_trace(0, refs)
    o.set_trace(0, refs)
    traced(g, o, 450)
    assert g.stats()["wt_sent"] == 0 and g.stats()["l1_hit"] == 1
    traced(g, o, 1200)
    same(g, o)
    assert g.stats()["wt_sent"] == 1 and g.stats()["wt_hit"] == 1


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_write_back_policies_and_drain(noc, oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, l1_write_back=1)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9)
    g, o = noc.Sim(p, tiling=(3, 2)), oracle_mod.OracleSim(p)
    traced(g, o, 3000)
    same(g, o)
    g.step(1000)                                   # the untraced loop as well
    o.step(1000)
    same(g, o)
    assert g.drain(100_000) == o.drain(100_000)
    same(g, o)
    assert g.stats()["wt_sent"] > 0


@pytest.mark.parametrize("tiling", [None, (4, 4)])
def test_write_back_mesh8(noc, oracle_mod, tiling):
    p = dict(I.MESH_8["params"])
    p.update(l1_write_back=1)
    g, o = noc.Sim(p, tiling=tiling), oracle_mod.OracleSim(p)
    traced(g, o, 1500)
    same(g, o)
    g.step(1500)
    o.step(1500)
    same(g, o)
    # fewer writes reach the L2 banks than under write-through
    q = dict(I.MESH_8["params"])
    w = oracle_mod.OracleSim(q)
    w.step(3000)
    assert g.stats()["wt_sent"] < w.stats()["wt_sent"]


def test_write_back_mesh64(noc, oracle_mod):
    p = I.mesh_64(2)
    p.update(l1_write_back=1)
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    g.step(1200)
    o.step(1200)
    same(g, o)


def test_write_back_instances_in_a_batch(noc, oracle_mod):
    pts = I.batch_design_points(10, seed=6, sides=(8, 16), period_lo=2, period_hi=10)
    for k, p in enumerate(pts):
        p.pop("design")
        if k % 2 == 1:
            p.update(l1_write_back=1)
    b = noc.Batch(pts, 1000, rect=8)
    b.run()
    for i, p in enumerate(pts):
        o = oracle_mod.OracleSim(p)
        o.step(1000)
        st = o.stats()
        g = b.stats(i)
        for k in ("injected", "ejected", "reply_rcvd", "l2lat_sum", "wt_sent"):
            assert g[k] == st[k], (i, k)
        assert b.state_hash(i) == o.state_hash(), i
