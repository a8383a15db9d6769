"""The centralized directory node (every LSPD directory message to one tile)
on the CUDA path against the oracle: every cycle's state hash, counters and
the full state, with drains, under both LSPD policies and two node positions."""
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
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


@pytest.mark.parametrize("policy,node", [(1, 14), (2, 14), (2, 0)])
def test_central_directory_parity(noc, oracle_mod, policy, node):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, dir_central=1, dir_tile=node)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9)
    g, o = noc.Sim(p, tiling=(3, 2)), oracle_mod.OracleSim(p)
    tg, to = g.step(3000, trace=True), o.step(3000, trace=True)
    assert (tg == to).all()
    same(g, o)
    g.step(1000)
    o.step(1000)
    same(g, o)
    assert g.drain(100_000) == o.drain(100_000)
    same(g, o)
    assert g.stats(node)["dir_search"] == g.stats()["dir_search"] > 0


def test_central_directory_hot_spot_overflows_identically(noc, oracle_mod):
    """4,096 cores sending every directory lookup to one tile: the node's
    service queue overflows -- the hot spot of the centralized organisation --
    at the same cycle on both sides."""
    p = I.mesh_64(1)
    p.update(policy=2, dir_central=1, dir_tile=64 * 32 + 32)
    o = oracle_mod.OracleSim(p)
    o.step(3000, check=False)
    code, cyc = o.error()
    assert code == 3 and 0 < cyc < 3000
    g = noc.Sim(p)
    g.step_async(3000)
    assert g.error() == (code, cyc)
