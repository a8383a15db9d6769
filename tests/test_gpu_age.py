"""The deflection-count age (age_mode 1: most deflections first, then inject
cycle, then source tile) on the CUDA path against the oracle: single-router
cases at centre, edge and corner routers, the link contents (ages included)
under load, every cycle's state hash in network and cache mode under the
three policies with drains, 64x64, the age and cycle limits, and age_mode
instances in a batch."""
import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu
N_, S_, E_, W_ = 0, 1, 2, 3


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def quiet(w, h, **over):
    cache = I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1, age_mode=1)
    p = I.sim_params(w, h, cache=cache, traf=I.traffic(period=0))
    p.update(over)
    return p


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


@pytest.mark.parametrize("here", [4, 1, 0])
def test_single_router_cases(noc, oracle_mod, here):
    rng = np.random.default_rng(7 + here)
    x, y = here % 3, here // 3
    ports = [p for p, ok in zip((N_, S_, E_, W_), (y > 0, y < 2, x < 2, x > 0)) if ok]
    for trial in range(25):
        p = quiet(3, 3)
        g, o = noc.Sim(p), oracle_mod.OracleSim(p)
        g.step(10)
        o.step(10)
        k = int(rng.integers(0, len(ports) + 1))
        used = rng.choice(ports, size=k, replace=False)
        srcs = rng.choice([r for r in range(9) if r != here], size=k, replace=False)
        for d, src in zip(used, srcs):
            f = dict(type="PROBE", src=int(src), dst=int(rng.integers(0, 9)),
                     inject=int(rng.integers(0, 4)), age=int(rng.integers(0, 3)))
            g.debug_link(here, int(d), f)
            o.debug_link(here, int(d), f)
        if rng.random() < 0.6:
            q = dict(type="PROBE", dst=int(rng.choice([r for r in range(9) if r != here])))
            g.debug_enqueue(here, 0, q)
            o.debug_enqueue(here, 0, q)
        g.step(1)
        o.step(1)
        assert (g.links() == o.links()).all(), trial
        same(g, o)


def test_conflict_and_limits(noc, oracle_mod):
    p = quiet(3, 3)
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    for s in (g, o):
        s.step(10)
        s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=0))
        s.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=7, age=2))
        s.step(1)
    lk = g.links()
    assert lk[4, E_][1] == 1 and lk[4, E_][7] == 2 and lk[4, N_][1] == 3 and lk[4, N_][7] == 1
    assert (lk == o.links()).all()
    traced(g, o, 5)
    same(g, o)
    # a flit deflected at age 4095: error 8 in that cycle on both sides
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    for s in (g, o):
        s.step(10)
        s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=4095))
        s.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=7, age=4095))
    g.step_async(1)
    o.step(1, check=False)
    assert g.error() == o.error() == (8, 10)
    # runs end at or before cycle 2^20
    g = noc.Sim(p)
    with pytest.raises(noc.NocError):
        g.step((1 << 20) + 1)
    with pytest.raises(noc.NocError):
        g.drain((1 << 20) + 1)
    with pytest.raises(noc.NocError):
        noc.Sim(quiet(3, 3)).debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=4096))


@pytest.mark.parametrize("tiling", [None, (2, 3)])
def test_network_load_links_and_hashes(noc, oracle_mod, tiling):
    traf = I.traffic(period=2, mode=I.MODE_NETWORK)
    cache = I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1, age_mode=1)
    p = I.sim_params(6, 6, seed=3, traf=traf, cache=cache)
    g, o = noc.Sim(p, tiling=tiling), oracle_mod.OracleSim(p)
    traced(g, o, 800)
    assert (g.links() == o.links()).all()
    assert g.links()[:, :, 7].max() >= 2
    same(g, o)
    g.step(700)                                    # the untraced loop as well
    o.step(700)
    assert (g.links() == o.links()).all()
    same(g, o)


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_cache_policies_and_drain(noc, oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, age_mode=1)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9)
    g, o = noc.Sim(p, tiling=(3, 2)), oracle_mod.OracleSim(p)
    traced(g, o, 2500)
    same(g, o)
    g.step(1000)
    o.step(1000)
    same(g, o)
    assert g.drain(100_000) == o.drain(100_000)
    same(g, o)


def test_mesh64_hotspot(noc, oracle_mod):
    p = I.mesh_64(1)
    p.update(age_mode=1)
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    g.step(1200)
    o.step(1200)
    same(g, o)
    assert (g.links() == o.links()).all()


def test_age_instances_in_a_batch(noc, oracle_mod):
    pts = I.batch_design_points(10, seed=8, sides=(8, 16), period_lo=2, period_hi=10)
    for k, p in enumerate(pts):
        p.pop("design")
        if k % 2 == 0:
            p.update(age_mode=1)
    b = noc.Batch(pts, 1000, rect=8)
    b.run()
    for i, p in enumerate(pts):
        o = oracle_mod.OracleSim(p)
        o.step(1000)
        st = o.stats()
        g = b.stats(i)
        for k in ("injected", "ejected", "deflections", "lat_sum", "l2lat_sum"):
            assert g[k] == st[k], (i, k)
        assert b.state_hash(i) == o.state_hash(), i
