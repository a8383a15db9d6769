"""The batch engine: every instance of a mixed batch (mesh sizes, loads,
address mixes, L2 policies, seeds) equals its own oracle run bit for bit, for
several CTA rectangle sizes and when the instances run in several memory
waves; and equals running the instance alone through the single-simulation
path."""
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("injected", "ejected", "deflections", "lat_sum", "lat_max", "refs", "l1_hit", "l1_miss",
        "l2_hit", "l2_miss", "req_made", "req_rcvd", "reply_sent", "reply_rcvd", "dir_search",
        "mem_req", "mem_write", "mem_wb", "wt_sent", "wt_hit", "trap", "redir", "migrations",
        "l2lat_sum", "l2lat_cnt", "cq_stall", "mm_stall", "mig_sent", "cycle")


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def small_points(n=20, cycles=1200, seed=3):
    pts = I.batch_design_points(n, seed=seed, sides=tuple(range(8, 41, 8)), period_lo=2,
                                period_hi=12)
    for p in pts:
        p.pop("design")
    return pts, cycles


def n_variant_groups(pts):
    """Kernel-variant groups among pts (the library's rule, pinned by
    tests/test_tune.py): each group runs in its own work-queue launches."""
    from paper_1508_03235_b300 import noc
    return len(set(noc.batch_groups(pts)))


@pytest.fixture(scope="module")
def oracle_results(oracle_mod):
    pts, cycles = small_points()
    res = []
    for p in pts:
        o = oracle_mod.OracleSim(p)
        o.step(cycles)
        st = o.stats()
        res.append((st, o.state_hash(), o.hist(0), o.hist(1)))
    return pts, cycles, res


@pytest.mark.parametrize("rect,strips,tmap", [(8, False, 0), (5, False, 1), (19, False, 2),
                                               (8, True, 2), (11, True, 0)])
def test_batch_matches_oracle(noc, oracle_results, rect, strips, tmap):
    pts, cycles, res = oracle_results
    b = noc.Batch(pts, cycles, rect=rect, strips=strips, thread_map=tmap)
    b.run()
    assert b.waves == n_variant_groups(pts)     # the pool holds every group at once
    for i, (st, h, h0, h1) in enumerate(res):
        g = b.stats(i)
        for k in KEYS:
            assert g[k] == st[k], (i, k)
        assert b.state_hash(i) == h, i
        assert (b.hist(i, 0) == h0).all() and (b.hist(i, 1) == h1).all()
    assert {p["policy"] for p in pts} == {0, 1, 2}


def test_batch_in_memory_waves(noc, oracle_results):
    pts, cycles, res = oracle_results
    import ctypes as C
    probe = noc.Batch(pts, cycles)
    need = noc.lib().noc_batch_min_bytes(probe._h)
    probe.close()
    b = noc.Batch(pts, cycles, pool_bytes=3 * need)
    b.run()
    assert b.waves > 2
    for i, (st, h, _, _) in enumerate(res):
        assert b.state_hash(i) == h, i


def test_batch_equals_one_at_a_time(noc):
    pts, cycles = small_points(n=6, cycles=900, seed=11)
    b = noc.Batch(pts, cycles)
    b.run()
    for i, p in enumerate(pts):
        s = noc.Sim(p)
        s.step(cycles)
        assert s.state_hash() == b.state_hash(i)
        assert s.stats() == b.stats(i)
