"""Seeded random configurations against the oracle: mesh shape, L2 policy,
way counts, queue sizes, traffic mix and period, every option (packets,
write-back, directory node, deflection-count age), CTA tiling and thread
order drawn together, so that combinations no hand-written case covers are
checked cycle by cycle (state hash), then after the plain loop and a drain."""
import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu

N_CASES = 64


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    w, h = int(rng.integers(1, 15)), int(rng.integers(1, 13))
    policy = int(rng.integers(0, 3))
    l1_ways, l2_ways = int(rng.integers(1, 9)), int(rng.integers(1, 17))
    l1_sets, l2_sets = int(rng.choice([4, 8, 16, 32])), int(rng.choice([8, 16, 64]))
    packets = int(rng.random() < 0.35)
    cache = I.cache_cfg()
    cache.update(l1_sets=l1_sets, l1_ways=l1_ways, l2_sets=l2_sets, l2_ways=l2_ways,
                 l1_miss_cycles=int(rng.integers(0, 6)), mem_latency=int(rng.integers(1, 120)),
                 mig_window=int(rng.integers(2, 12)), mig_threshold=int(rng.integers(1, 4)),
                 core_q=int(rng.integers(1, 9)), svc_q=2048, mem_q=256,
                 fwd_entries=int(rng.integers(1, 5)), packet_mode=packets,
                 rob_entries=int(rng.integers(1, 9)),
                 dir_central=int(rng.random() < 0.25), dir_tile=int(rng.integers(0, w * h)),
                 l1_write_back=int(rng.random() < 0.35), age_mode=int(rng.random() < 0.35))
    fr = rng.dirichlet((2, 2, 1))
    traf = I.traffic(period=int(rng.integers(1, 12)), write=float(rng.uniform(0, 0.6)),
                     priv=float(fr[0]), shared=float(fr[1]), priv_kb=int(rng.choice([1, 4, 16])),
                     shared_mb=0)
    traf.update(shared_lines=int(rng.integers(50, 2000)))
    p = I.sim_params(w, h, policy=policy, cache=cache, traf=traf, seed=int(rng.integers(1, 1 << 30)))
    gx, gy = int(rng.integers(1, w + 1)), int(rng.integers(1, h + 1))
    while -(-w // gx) * -(-h // gy) > 384:
        gx, gy = gx + 1, gy + 1
    return p, (min(gx, w), min(gy, h)), int(rng.integers(0, 3))


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_configuration(noc, oracle_mod, seed):
    p, tiling, tmap = draw(seed)
    g = noc.Sim(p, tiling=tiling, thread_map=tmap)
    o = oracle_mod.OracleSim(p)
    n1 = 800
    to = o.step(n1, trace=True, check=False)
    code, cyc = o.error()
    if code:
        # a configuration that overflows a queue: the same error at the same cycle
        g.step_async(n1)
        assert g.error() == (code, cyc), (p, tiling, tmap)
        return
    tg = g.step(n1, trace=True)
    bad = np.nonzero(tg != to)[0]
    assert len(bad) == 0, (f"first per-cycle hash mismatch at cycle {bad[0]}", p, tiling, tmap)
    g.step(700)
    o.step(700, check=False)
    if o.error()[0]:
        return
    assert g.state_hash() == o.state_hash(), (p, tiling, tmap)
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (k, p, tiling, tmap)
    try:
        taken = o.drain(100_000)
    except Exception:
        return
    assert g.drain(100_000) == taken
    assert g.state_hash() == o.state_hash()


@pytest.mark.parametrize("seed", range(0, N_CASES, 2))
def test_random_configuration_two_tiles_per_thread(noc, oracle_mod, seed):
    """The same draws through the two-tile loop (plain steps only), switching
    to the one-tile loop midway and back: every end state equal to the
    oracle's, and a queue overflow at the same cycle."""
    p, tiling, tmap = draw(seed)
    # rectangles of up to 512 tiles hold two per thread; keep the draw's shape
    g = noc.Sim(p, tiling=tiling, thread_map=tmap, tiles_per_thread=2)
    o = oracle_mod.OracleSim(p)
    for k, n in ((2, 600), (1, 300), (2, 600)):
        g.set_tiles_per_thread(k)
        o.step(n, check=False)
        code, cyc = o.error()
        if code:
            g.step_async(n)
            assert g.error() == (code, cyc), (p, tiling, tmap)
            return
        g.step(n)
        assert g.tiles_per_thread() == k
        assert g.state_hash() == o.state_hash(), (k, p, tiling, tmap)
    gs, os_ = g.stats(), o.stats()
    for key, v in os_.items():
        if key in gs:
            assert gs[key] == v, (key, p, tiling, tmap)
    for w in (0, 1):
        assert (g.hist(w) == o.hist(w)).all()
