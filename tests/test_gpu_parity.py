"""Parity of the CUDA path (through the C ABI) with the oracle, bit for bit:
per-cycle state hashes, counters, latency histograms, full state hashes and
element-by-element state, on the named workloads, ragged meshes, every CTA
tiling and every L2 policy."""
import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu

COUNTERS = ("injected", "ejected", "in_flight", "deflections", "lat_sum", "lat_max", "refs",
            "l1_hit", "l1_miss", "l2_hit", "l2_miss", "req_made", "req_rcvd", "reply_sent",
            "reply_rcvd", "dir_search", "mem_req", "mem_write", "mem_wb", "wt_sent", "wt_hit",
            "trap", "redir", "migrations", "l2lat_sum", "l2lat_cnt", "cq_stall", "mm_stall",
            "mig_sent", "cycle")


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def pair(noc, oracle_mod, params, tiling=None):
    return noc.Sim(params, tiling=tiling), oracle_mod.OracleSim(params)


def assert_same(g, o, hist=True):
    gs, os_ = g.stats(), o.stats()
    for k in COUNTERS:
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    if hist:
        for w in (0, 1):
            assert (g.hist(w) == o.hist(w)).all(), f"histogram {w}"
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


def run_traced(g, o, n):
    tg = g.step(n, trace=True)
    to = o.step(n, trace=True)
    bad = np.nonzero(tg != to)[0]
    assert len(bad) == 0, f"first per-cycle hash mismatch at cycle {o.cycle - n + bad[0]}"


# --------------------------------------------------------------------------
def test_mesh8_every_cycle(noc, oracle_mod):
    g, o = pair(noc, oracle_mod, I.MESH_8["params"])
    run_traced(g, o, 3000)
    assert_same(g, o)
    for k in range(3):                   # several launches in a row
        run_traced(g, o, 700 + 31 * k)
    assert_same(g, o)


def test_mesh8_full_length(noc, oracle_mod):
    g, o = pair(noc, oracle_mod, I.MESH_8["params"])
    g.step(I.MESH_8["cycles"])
    o.step(I.MESH_8["cycles"])
    assert_same(g, o)


@pytest.mark.parametrize("tiling", [(1, 1), (2, 2), (8, 8), (3, 5), (8, 1), (1, 8)])
def test_tilings_hash_identically(noc, oracle_mod, tiling):
    g, o = pair(noc, oracle_mod, I.MESH_8["params"], tiling=tiling)
    run_traced(g, o, 1500)
    assert_same(g, o)
    assert g.tiling() == tiling


@pytest.mark.parametrize("thread_map", [1, 2])
@pytest.mark.parametrize("tiling", [(1, 1), (3, 2), (2, 5), (13, 1)])
def test_thread_maps(noc, oracle_mod, thread_map, tiling):
    """Row-major and column-major tile-to-thread orders (the autotuner's other
    choices) on square, ragged and thin rectangles: the traced loop (its
    perimeter-warp barrier then spans every warp), the plain loop and a
    drain."""
    cache = I.cache_cfg(l2_kb=64, svc_q=512)
    p = I.sim_params(13, 11, policy=2 if tiling[0] % 2 else 0, seed=4, cache=cache,
                     traf=I.traffic(period=3, priv=0.4, shared=0.5, shared_mb=1))
    g = noc.Sim(p, tiling=tiling, thread_map=thread_map)
    o = oracle_mod.OracleSim(p)
    assert g.thread_map() == thread_map
    run_traced(g, o, 600)
    assert_same(g, o)
    g.step(900)
    o.step(900)
    assert_same(g, o)
    assert g.drain(100_000) == o.drain(100_000)
    assert_same(g, o)


@pytest.mark.parametrize("tiling", [(1, 1), (2, 2), (8, 8), (3, 5), (8, 1), (1, 8), (4, 3)])
def test_tilings_untraced(noc, oracle_mod, tiling):
    """The untraced cycle loop (per-warp cycle flags, no CTA barrier per cycle)
    on every shape of rectangle, down to one tile per CTA, over several
    launches."""
    g, o = pair(noc, oracle_mod, I.MESH_8["params"], tiling=tiling)
    for n in (1, 2, 700, 333):
        g.step(n)
        o.step(n)
        assert_same(g, o)


@pytest.mark.parametrize("policy", [1, 2])
def test_lspd_policies_mesh8(noc, oracle_mod, policy):
    p = I.sim_params(8, 8, policy=policy, seed=1)
    g, o = pair(noc, oracle_mod, p)
    run_traced(g, o, 2500)
    assert_same(g, o)


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_heavy_sharing_and_drain(noc, oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9)
    g, o = pair(noc, oracle_mod, p, tiling=(3, 2))
    run_traced(g, o, 4000)
    assert g.drain(100_000) == o.drain(100_000)
    assert_same(g, o)
    if policy == 2:
        assert g.stats()["migrations"] > 0
    # the state after a drain is a fixed point
    h = g.dyn_hash()
    run_traced(g, o, 40)
    assert g.dyn_hash() == h


@pytest.mark.parametrize("w,h,tiling", [(13, 7, (4, 3)), (1, 1, None), (1, 17, None),
                                         (17, 1, (5, 1)), (31, 29, (7, 6))])
def test_ragged_meshes(noc, oracle_mod, w, h, tiling):
    p = I.sim_params(w, h, seed=5, traf=I.traffic(period=3, priv=0.5, shared=0.4))
    g, o = pair(noc, oracle_mod, p, tiling=tiling)
    run_traced(g, o, 1200)
    assert_same(g, o)
    g2 = noc.Sim(p, tiling=tiling)
    g2.step(1200)
    assert_same(g2, o)


def test_mesh64_hotspot(noc, oracle_mod):
    g, o = pair(noc, oracle_mod, I.mesh_64(1))
    run_traced(g, o, 1500)
    assert_same(g, o)
    g2 = noc.Sim(I.mesh_64(1), tiling=(16, 16))
    g2.step(1500)
    assert g2.state_hash() == o.state_hash()


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_mesh64_seeds_prefix(noc, oracle_mod, seed):
    g, o = pair(noc, oracle_mod, I.mesh_64(seed))
    g.step(2000)
    o.step(2000)
    assert_same(g, o)


@pytest.mark.parametrize("period", [10, 2])
def test_mesh208_full_size_prefix(noc, oracle_mod, period):
    """The 208x208 mesh in the bench's launch configuration (the tuned tiling
    and tile-to-thread order): every cycle of a prefix, then the full state
    after the plain cycle loop."""
    from paper_1508_03235_b300 import tune
    p = I.mesh_208(period)
    tiling, tmap = tune.cached_tiling(p), tune.cached_thread_map(p)
    g = noc.Sim(p, tiling=tiling, thread_map=tmap)
    o = oracle_mod.OracleSim(p)
    run_traced(g, o, 160)
    assert_same(g, o)
    g2 = noc.Sim(p, tiling=tiling, thread_map=tmap)
    g2.step(100)
    g2.step(60)
    assert_same(g2, o)


def test_network_mode(noc, oracle_mod):
    traf = I.traffic(period=2, mode=I.MODE_NETWORK)
    p = I.sim_params(12, 10, seed=3, traf=traf, cache=I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1,
                                                                   l2_ways=1))
    g, o = pair(noc, oracle_mod, p, tiling=(3, 2))
    run_traced(g, o, 800)
    assert (g.links() == o.links()).all()
    assert_same(g, o)


def test_trace_mode_timelines(noc, oracle_mod):
    p = I.sim_params(3, 3, traf=I.traffic(period=10, mode=I.MODE_TRACE))
    g, o = pair(noc, oracle_mod, p)
    for s in (g, o):
        s.set_trace(0, [8, 17, 8 | (1 << 31)])
        s.set_trace(4, [13, 4, 13 | (1 << 31)])
    run_traced(g, o, 400)
    assert_same(g, o)
    assert g.stats()["l2lat_sum"] == o.stats()["l2lat_sum"]


def test_debug_links_and_queues(noc, oracle_mod):
    p = I.sim_params(3, 3, cache=I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1),
                     traf=I.traffic(period=0))
    g, o = pair(noc, oracle_mod, p)
    for s in (g, o):
        s.step(10)
        s.debug_link(4, 3, dict(type="PROBE", src=3, dst=5, inject=5))
        s.debug_link(4, 0, dict(type="PROBE", src=1, dst=5, inject=7))
        s.debug_enqueue(4, 0, dict(type="PROBE", dst=0))
        s.debug_enqueue(2, 1, dict(type="PROBE", dst=6))
    for _ in range(8):
        g.step(1)
        o.step(1)
        assert (g.links() == o.links()).all()
    assert_same(g, o)


def canonical_core(c):
    busy, wait, om = c["fsm"] != 0, c["fsm"] == 1, c["om_kind"] != 0
    mem = c["om_kind"] in (3, 4)
    return (c["next_ref"], c["fsm"], c["fsm_line"] if busy else 0, c["fsm_write"] if busy else 0,
            c["fsm_timer"] if wait else 0, c["fsm_start"] if wait else 0, c["om_kind"],
            c["om_line"] if om else 0, c["om_write"] if om else 0, c["om_start"] if om else 0,
            c["om_timer"] if mem else 0, c["om_epoch"] if c["om_kind"] == 3 else 0, c["epoch"],
            c["cq_len"], c["sq_len"], c["mq_len"], c["fwd_n"])


@pytest.mark.parametrize("policy", [0, 2])
def test_element_by_element_state(noc, oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=4, l2_kb=8, l2_ways=8, mig_window=4, mig_threshold=2)
    traf = I.traffic(period=4, priv=0.4, shared=0.5, shared_mb=0)
    traf.update(shared_lines=500)
    p = I.sim_params(5, 4, policy=policy, cache=cache, traf=traf, seed=21)
    g, o = pair(noc, oracle_mod, p, tiling=(2, 2))
    g.step(1777)
    o.step(1777)
    assert (g.links() == o.links()).all()
    for t in range(20):
        assert canonical_core(g.core(t)) == canonical_core(o.core(t)), t
        for which in (1, 2):
            assert (g.cache(t, which) == o.cache(t, which)).all(), (t, which)
        gs, os_ = g.stats(t), o.stats(t)
        for k in COUNTERS:
            if k not in ("in_flight", "cycle"):
                assert gs[k] == os_[k], (t, k)
    if policy:
        for line in range(0, p["remote_lines"] + 600, 997):
            assert g.dir_get(line) == o.dir_get(line)
    assert_same(g, o)


def test_overflow_error_parity(noc, oracle_mod):
    p = I.sim_params(8, 8, seed=1, cache=I.cache_cfg(svc_q=1),
                     traf=I.traffic(period=1, priv=0.0, shared=1.0, hot=1.0, hot_side=1,
                                    shared_mb=1))
    o = oracle_mod.OracleSim(p)
    o.step(20_000, check=False)
    code, cyc = o.error()
    assert code == 3
    g = noc.Sim(p, tiling=(2, 2))
    g.step_async(cyc + 50)
    assert g.error() == (code, cyc)
    with pytest.raises(noc.NocError):
        g.step(10)


def test_bounded_wait_times_out(noc):
    """A CTA that never publishes its cycle: its neighbours' waits run out and
    the step ends with NOC_ERR_TIMEOUT; the context stays usable."""
    import time
    g = noc.Sim(I.MESH_8["params"], tiling=(2, 2))
    g.wait_limit(50_000_000, silent_cta=3)
    t = time.time()
    g.step_async(1000)
    code, cyc = g.error()
    assert code == 4 and 0 <= cyc < 1000
    assert time.time() - t < 20
    # the device still works
    h = noc.Sim(I.MESH_8["params"])
    h.step(100)
    assert h.stats()["cycle"] == 100


def test_general_way_bounds(noc, oracle_mod):
    """8-way L1 and 16-way L2 run the general (16, 16) kernel variant."""
    cache = I.cache_cfg(l1_kb=4, l1_ways=8, l2_kb=16, l2_ways=16, mig_window=6, mig_threshold=3)
    traf = I.traffic(period=3, priv=0.4, shared=0.5, shared_mb=0)
    traf.update(shared_lines=900)
    for policy in (0, 2):
        p = I.sim_params(7, 6, policy=policy, cache=cache, traf=traf, seed=13)
        g, o = pair(noc, oracle_mod, p, tiling=(2, 2))
        run_traced(g, o, 1500)
        assert_same(g, o)


@pytest.mark.parametrize("policy,l1_ways,l2_ways", [(0, 3, 6), (2, 5, 12), (1, 1, 7)])
def test_ways_that_are_not_powers_of_two(noc, oracle_mod, policy, l1_ways, l2_ways):
    """Any way count 1..16 (the cache-set code ranks ways up to ways - 1, so
    nothing assumes a power of two); these run on the general and base kernels
    and their way-bound classes."""
    cache = I.cache_cfg(l1_kb=3 * l1_ways, l1_ways=l1_ways, l2_kb=6 * l2_ways, l2_ways=l2_ways,
                        mig_window=4, mig_threshold=2, svc_q=512)
    traf = I.traffic(period=3, priv=0.4, shared=0.5, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=400)
    p = I.sim_params(9, 7, policy=policy, cache=cache, traf=traf, seed=3)
    g, o = pair(noc, oracle_mod, p, tiling=(3, 2))
    run_traced(g, o, 2000)
    assert_same(g, o)
    g.step(1500)
    o.step(1500)
    assert_same(g, o)
    assert g.stats()["l1_hit"] > 0 and g.stats()["l2_hit"] > 0
