"""The plain loop with two tiles per thread (the capacity loop, for meshes
beyond one co-resident launch of one thread per tile), forced on meshes of
every shape against the oracle, bit for bit: every L2 policy and option, the
three thread orders, ragged and thin rectangles, several launches in a row;
the traced loop and drains are refused on it; its bounded waits time out
like the one-tile loop's."""
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


def assert_same(g, o):
    gs, os_ = g.stats(), o.stats()
    for k in COUNTERS:
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    for w in (0, 1):
        assert (g.hist(w) == o.hist(w)).all(), f"histogram {w}"
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


def busy_params(w, h, policy, seed, **opts):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=8, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, **opts)
    traf = I.traffic(period=3, priv=0.35, shared=0.5, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=400, remote_lines=20_000)
    return I.sim_params(w, h, policy=policy, cache=cache, traf=traf, seed=seed)


CASES = {
    "interleaved_mesh8": (dict(I.MESH_8["params"]), (2, 2), 0),
    "lspd_ragged": (busy_params(13, 11, 1, 3), (3, 2), 1),
    "migrate_columns": (busy_params(12, 10, 2, 4), (2, 3), 2),
    "packets_perimeter": (busy_params(9, 9, 2, 5, packet_mode=1), (2, 2), 0),
    "write_back_thin": (busy_params(17, 5, 0, 6, l1_write_back=1), (1, 5), 1),
    "age_dir_node": (busy_params(10, 8, 1, 7, age_mode=1, dir_central=1, dir_tile=33), (2, 2), 2),
    "one_rect": (busy_params(11, 9, 2, 8), (1, 1), 0),
    "one_tile_rects": (busy_params(6, 5, 0, 9), (6, 5), 1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_two_tiles_per_thread_match_oracle(noc, oracle_mod, name):
    p, tiling, tmap = CASES[name]
    g = noc.Sim(p, tiling=tiling, thread_map=tmap, tiles_per_thread=2)
    o = oracle_mod.OracleSim(p)
    for n in (1, 700, 333, 1500):         # several launches, each resuming the last
        g.step(n)
        o.step(n)
        assert_same(g, o)
    assert g.tiles_per_thread() == 2
    assert g.variant()["loop"] == "plain, two tiles per thread"
    assert (g.links() == o.links()).all()


def test_traced_loop_and_drain_are_refused(noc):
    g = noc.Sim(I.MESH_8["params"], tiles_per_thread=2)
    g.step(10)
    with pytest.raises(noc.NocError) as e:
        g.step(10, trace=True)
    assert e.value.code == 1
    with pytest.raises(noc.NocError):
        g.drain(100)
    # back to one tile per thread: both work again, from the same state
    g.set_tiles_per_thread(1)
    g.step(10, trace=True)
    assert g.tiles_per_thread() == 1


def test_switching_between_loops_mid_run(noc, oracle_mod):
    p = busy_params(12, 9, 2, 12)
    g = noc.Sim(p, tiling=(2, 2))
    o = oracle_mod.OracleSim(p)
    for k, n in ((1, 400), (2, 500), (1, 300), (2, 600)):
        g.set_tiles_per_thread(k)
        g.step(n)
        o.step(n)
        assert g.tiles_per_thread() == k
    assert_same(g, o)


def test_bounded_wait_times_out(noc):
    import time
    g = noc.Sim(I.MESH_8["params"], tiling=(2, 2), tiles_per_thread=2)
    g.wait_limit(50_000_000, silent_cta=3)
    t = time.time()
    g.step_async(1000)
    code, cyc = g.error()
    assert code == 4 and 0 <= cyc < 1000
    assert time.time() - t < 20
