"""Every build of the cycle kernel the library ships, against the oracle, bit
for bit, on configurations that evict all the time.

The library compiles the cycle kernel once per way-bound class, (L1, L2) ways
(4, 8), (4, 16) and (16, 16), and per specialisation: "interleaved",
"lspd-local" and "lspd-migrate" (one L2 policy in cache mode with exactly the
class's way counts and no option), "base" (every policy, no packet /
write-back / directory-node / age option) and "general" (everything); the
traced loop (per-cycle hash record) and the draining loop are general builds
of each class; the batch kernel comes in the same fifteen builds.  Each case here is built so that its configuration selects
one build, asserts through noc_last_variant / noc_batch_variant that this
build ran, and compares counters, both histograms and the dynamic and full
state hashes with the oracle.  The caches are tiny (16 lines of L1, 16 of L2
per tile) against a 32-line private working set, a 300-line shared region
and a 4,000-line remote one, so L1 and L2 victims, write-throughs, dirty L2
write-backs and (LSPD policies) directory deletions happen every few
cycles."""
import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu

BOUNDS = ((4, 8), (4, 16), (16, 16))
KINDS = ("interleaved", "lspd-local", "lspd-migrate", "base", "general")
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


def variant_params(kind, bounds, w=7, h=6, seed=5):
    """A configuration that runs on build (kind, bounds)."""
    opts, policy = {}, 0
    if kind in ("interleaved", "lspd-local", "lspd-migrate"):
        l1w, l2w = bounds
        policy = ("interleaved", "lspd-local", "lspd-migrate").index(kind)
    elif kind == "base":
        l1w, l2w = {(4, 8): (3, 6), (4, 16): (4, 12), (16, 16): (8, 16)}[bounds]
        policy = {(4, 8): 1, (4, 16): 2, (16, 16): 2}[bounds]
    else:
        l1w, l2w = {(4, 8): (4, 8), (4, 16): (2, 16), (16, 16): (16, 16)}[bounds]
        policy, opts = {(4, 8): (2, dict(packet_mode=1)),
                        (4, 16): (0, dict(l1_write_back=1)),
                        (16, 16): (1, dict(age_mode=1, dir_central=1, dir_tile=20))}[bounds]
    cache = I.cache_cfg(l1_ways=l1w, l2_ways=l2w, mig_window=4, mig_threshold=2, svc_q=512, **opts)
    cache.update(l1_sets=max(1, 16 // l1w), l2_sets=max(1, 16 // l2w))
    traf = I.traffic(period=2, write=0.35, priv=0.35, shared=0.35, priv_kb=2, shared_mb=0)
    traf.update(shared_lines=300, remote_lines=4_000)
    return I.sim_params(w, h, policy=policy, cache=cache, traf=traf, seed=seed)


def assert_same(g, o):
    gs, os_ = g.stats(), o.stats()
    for k in COUNTERS:
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    for w in (0, 1):
        assert (g.hist(w) == o.hist(w)).all(), f"histogram {w}"
    assert g.dyn_hash() == o.dyn_hash()
    assert g.state_hash() == o.state_hash()


def assert_busy(st, lspd):
    """The run exercised victims and write traffic, not just hits."""
    assert st["l1_miss"] > 1000 and st["l2_miss"] > 500, st
    assert st["mem_wb"] > 20 and st["wt_sent"] + st["mem_wb"] > 100, st
    if lspd:
        assert st["dir_search"] > 500, st


@pytest.mark.parametrize("bounds", BOUNDS, ids=lambda b: f"{b[0]}x{b[1]}")
@pytest.mark.parametrize("kind", KINDS)
def test_plain_traced_and_draining_builds(noc, oracle_mod, kind, bounds):
    p = variant_params(kind, bounds)
    g = noc.Sim(p, tiling=(2, 2))
    o = oracle_mod.OracleSim(p)
    g.step(2500)
    o.step(2500)
    assert g.variant() == dict(loop="plain", kind=kind, bounds=bounds)
    assert g.launch_bound() == 320            # small CTAs: the narrow build
    g.step(1500)                              # a second launch continues the first
    o.step(1500)
    assert g.variant() == dict(loop="plain", kind=kind, bounds=bounds)
    assert_same(g, o)
    assert_busy(o.stats(), p["policy"] != 0)
    # the traced loop: the dynamic hash of every cycle
    tg, to = g.step(400, trace=True), o.step(400, trace=True)
    assert g.variant() == dict(loop="traced", kind="general", bounds=bounds)
    bad = np.nonzero(tg != to)[0]
    assert len(bad) == 0, f"first per-cycle hash mismatch at cycle {o.cycle - 400 + bad[0]}"
    # the draining loop, to quiescence
    assert g.drain(200_000) == o.drain(200_000)
    assert g.variant() == dict(loop="traced", kind="general", bounds=bounds)
    assert_same(g, o)


@pytest.mark.parametrize("bounds", BOUNDS, ids=lambda b: f"{b[0]}x{b[1]}")
def test_batch_builds(noc, oracle_mod, bounds):
    """One batch per way class, holding instances of all five kinds (two
    interleaved ones, one spanning 3 x 2 rectangles): each instance runs on
    its kind's batch build of that class and equals its oracle run."""
    pts = [variant_params(k, bounds, seed=20 + j) for j, k in enumerate(KINDS)]
    pts.append(variant_params("interleaved", bounds, w=11, h=7, seed=30))
    cycles = 3000
    b = noc.Batch(pts, cycles, rect=4)
    b.run()
    for i, p in enumerate(pts):
        kind = KINDS[i] if i < len(KINDS) else "interleaved"
        assert b.variant(i) == dict(kind=kind, bounds=bounds), i
        o = oracle_mod.OracleSim(p)
        o.step(cycles)
        gs, os_ = b.stats(i), o.stats()
        for k in COUNTERS:
            assert gs[k] == os_[k], (i, k, gs[k], os_[k])
        assert b.state_hash(i) == o.state_hash(), i
        for w in (0, 1):
            assert (b.hist(i, w) == o.hist(w)).all(), (i, w)
        assert_busy(os_, p["policy"] != 0)
        o.close()
    b.close()


@pytest.mark.parametrize("mesh,launch_bound", [((19, 18), 384), ((21, 21), 448)],
                         ids=("384-thread build", "448-thread build"))
@pytest.mark.parametrize("bounds", BOUNDS, ids=lambda b: f"{b[0]}x{b[1]}")
@pytest.mark.parametrize("kind", KINDS)
def test_wide_plain_builds(noc, oracle_mod, kind, bounds, mesh, launch_bound):
    """The plain loop's builds for CTAs of more than 320 threads: a 19 x 18
    mesh in one CTA (342 tiles) runs on the build for up to 384 threads, a
    21 x 21 mesh (441 tiles, 14 warps) on the one for up to 448 (128
    registers a thread); two launches each, against the oracle."""
    p = variant_params(kind, bounds, w=mesh[0], h=mesh[1], seed=7)
    if p.get("dir_central"):
        p["dir_tile"] = 200
    g = noc.Sim(p, tiling=(1, 1))
    o = oracle_mod.OracleSim(p)
    for n in (1200, 800):
        g.step(n)
        o.step(n)
        assert g.variant() == dict(loop="plain", kind=kind, bounds=bounds)
        assert g.launch_bound() == launch_bound
    assert_same(g, o)
