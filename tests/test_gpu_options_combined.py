"""Every option beyond the paper's workloads at once -- multi-flit packets
with reorder buffers, the L1 write-back policy, the centralized directory node
and the deflection-count age -- on the general kernel variant against the
oracle, under each L2 policy and thread order: every cycle's state hash,
counters, histograms, full state and a drain."""
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


def same(g, o):
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (k, gs[k], v)
    for w in (0, 1):
        assert (g.hist(w) == o.hist(w)).all()
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


@pytest.mark.parametrize("policy,thread_map", [(0, 0), (1, 2), (2, 1)])
def test_all_options_at_once(noc, oracle_mod, policy, thread_map):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=1024, packet_mode=1, rob_entries=8, dir_central=1, dir_tile=17,
                        l1_write_back=1, age_mode=1)
    traf = I.traffic(period=3, write=0.35, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(7, 5, policy=policy, cache=cache, traf=traf, seed=12)
    g = noc.Sim(p, tiling=(3, 2), thread_map=thread_map)
    o = oracle_mod.OracleSim(p)
    tg, to = g.step(2500, trace=True), o.step(2500, trace=True)
    bad = np.nonzero(tg != to)[0]
    assert len(bad) == 0, f"first per-cycle hash mismatch at cycle {bad[0]}"
    same(g, o)
    g.step(1500)
    o.step(1500)
    same(g, o)
    assert g.drain(200_000) == o.drain(200_000)
    same(g, o)
    st = g.stats()
    assert st["wt_sent"] > 0 and st["deflections"] > 0
    if policy:
        assert g.stats(17)["dir_search"] == st["dir_search"] > 0
