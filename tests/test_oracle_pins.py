"""Pins of the oracle against facts fixed outside it: a library generator,
closed forms, brute force on tiny inputs and hand-worked timelines of the
paper's rules.  No expected value here comes from either simulator."""
import os
from collections import Counter, OrderedDict

import numpy as np
import pytest

from paper_1508_03235_b300 import inputs as I

N_, S_, E_, W_ = 0, 1, 2, 3


def quiet_params(w, h, policy=0, **over):
    """A mesh with no reference stream (period 0): flits come from the test."""
    cache = I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1)
    traf = I.traffic(period=0)
    p = I.sim_params(w, h, policy=policy, cache=cache, traf=traf)
    p.update(over)
    return p


def trace_params(w, h, policy=0, period=200, cache=None, **over):
    traf = I.traffic(period=period, mode=I.MODE_TRACE)
    p = I.sim_params(w, h, policy=policy, cache=cache or I.cache_cfg(), traf=traf)
    p.update(over)
    return p


# --------------------------------------------------------------------------
# Philox4x64-10 against numpy's implementation of the same published generator
def test_philox_matches_numpy(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        # numpy increments its 256-bit counter before each block
        c = sum(v << (64 * i) for i, v in enumerate(ctr)) - 1
        c %= 2**256
        prev = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
        bg = np.random.Philox(counter=prev, key=key)
        want = bg.random_raw(4)
        got = oracle_mod.philox4x64_10(ctr, key)
        assert [int(x) for x in got] == [int(x) for x in want]
    # the counter layout the model uses: (ref, core, stream, 0), key (seed, 'NOC')
    bg = np.random.Philox(counter=[2, 5, 0, 0], key=[7, 0x4E4F43])
    assert [int(x) for x in oracle_mod.philox4x64_10([3, 5, 0, 0], [7, 0x4E4F43])] == \
        [int(x) for x in bg.random_raw(4)]


def test_mix64_published_vector(oracle_mod):
    # splitmix64 seeded with 0: the generator adds the golden gamma, then
    # applies the finaliser; its first outputs are published test values
    g = 0x9E3779B97F4A7C15
    assert oracle_mod.mix64(g) == 0xE220A8397B1DCDAF
    assert oracle_mod.mix64((2 * g) % 2**64) == 0x6E789E6AA1B965F4


# --------------------------------------------------------------------------
# routing: a lone flit follows X then Y and takes |dx|+|dy| cycles (Sec. 4.2)
def test_lone_flit_xy_all_pairs(oracle_mod):
    W, H = 4, 3
    for src in range(W * H):
        for dst in range(W * H):
            if src == dst:
                continue
            s = oracle_mod.OracleSim(quiet_params(W, H))
            s.debug_enqueue(src, 0, dict(type="PROBE", dst=dst))
            hops = abs(src % W - dst % W) + abs(src // W - dst // W)
            ports = []
            for _ in range(hops):
                s.step(1)
                lk = s.links()
                on = np.argwhere(lk[:, :, 0] != 0)
                assert len(on) == 1
                ports.append(int(on[0][1]))
            s.step(1)
            st = s.stats()
            assert st["ejected"] == 1 and st["deflections"] == 0
            assert st["lat_sum"] == hops
            nx = abs(src % W - dst % W)
            assert all(p in (E_, W_) for p in ports[:nx])
            assert all(p in (N_, S_) for p in ports[nx:])


# --------------------------------------------------------------------------
# arbitration: oldest first, lower source on ties; loser deflected to the
# first free port of N, S, E, W (Sec. 4.3)
@pytest.mark.parametrize("inj_a,inj_b,winner", [(5, 7, "A"), (5, 5, "B")])
def test_two_flit_conflict(oracle_mod, inj_a, inj_b, winner):
    s = oracle_mod.OracleSim(quiet_params(3, 3))
    s.step(10)
    # A from the west neighbour (tile 3), B from the north neighbour (tile 1);
    # both are addressed to tile 5 = (2,1) and both want port E at tile 4
    s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=inj_a))
    s.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=inj_b))
    s.step(1)
    lk = s.links()
    east, north = lk[4, E_], lk[4, N_]
    win_src = 3 if winner == "A" else 1
    lose_src = 1 if winner == "A" else 3
    assert east[1] == win_src and north[1] == lose_src
    assert s.stats()["deflections"] == 1
    s.step(5)
    st = s.stats()
    assert st["ejected"] == 2 and st["in_flight"] == 0
    # winner: one hop (cycle 11); loser: N, then E, then S (cycle 13)
    inj_w = inj_a if winner == "A" else inj_b
    inj_l = inj_b if winner == "A" else inj_a
    assert st["lat_sum"] == (11 - inj_w) + (13 - inj_l)


def test_eject_priority_and_deflect_at_destination(oracle_mod):
    s = oracle_mod.OracleSim(quiet_params(3, 3))
    s.step(10)
    s.debug_link(4, W_, dict(type="PROBE", src=3, dst=4, inject=5))
    s.debug_link(4, N_, dict(type="PROBE", src=1, dst=4, inject=7))
    s.step(1)
    st = s.stats()
    assert st["ejected"] == 1 and st["lat_sum"] == 5 and st["deflections"] == 1
    assert s.links()[4, N_][1] == 1      # the younger one went back north
    s.step(2)
    st = s.stats()
    assert st["ejected"] == 2 and st["lat_sum"] == 5 + (12 - 7)


def test_no_injection_when_inputs_full(oracle_mod):
    s = oracle_mod.OracleSim(quiet_params(3, 3))
    s.step(10)
    s.debug_enqueue(4, 0, dict(type="PROBE", dst=0))
    # four flits pass through tile 4 (none addressed to it)
    s.debug_link(4, N_, dict(type="PROBE", src=1, dst=7, inject=3))
    s.debug_link(4, S_, dict(type="PROBE", src=7, dst=1, inject=3))
    s.debug_link(4, E_, dict(type="PROBE", src=5, dst=3, inject=3))
    s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=3))
    s.step(1)
    assert s.core(4)["cq_len"] == 1
    s.step(1)
    assert s.core(4)["cq_len"] == 0
    # corner tile 0 (two ports) with both inputs busy
    s2 = oracle_mod.OracleSim(quiet_params(3, 3))
    s2.step(4)
    s2.debug_enqueue(0, 0, dict(type="PROBE", dst=8))
    s2.debug_link(0, E_, dict(type="PROBE", src=1, dst=3, inject=1))
    s2.debug_link(0, S_, dict(type="PROBE", src=3, dst=1, inject=1))
    s2.step(1)
    assert s2.core(0)["cq_len"] == 1


# --------------------------------------------------------------------------
# invariants under load (network-only traffic)
def net_params(w, h, period, seed=3):
    traf = I.traffic(period=period, mode=I.MODE_NETWORK)
    cache = I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1)
    return I.sim_params(w, h, seed=seed, traf=traf, cache=cache)


def test_conservation_and_oldest_never_deflected(oracle_mod):
    W = H = 6
    s = oracle_mod.OracleSim(net_params(W, H, period=2))
    nbr = {N_: -W, S_: W, E_: 1, W_: -1}
    max_in_flight = 0
    for _ in range(400):
        lk = s.links()
        valid = np.argwhere(lk[:, :, 0] != 0)
        st = s.stats()
        assert len(valid) == st["injected"] - st["ejected"]          # conservation
        assert len(valid) <= 2 * (W * (H - 1) + H * (W - 1))         # one per directed link
        max_in_flight = max(max_in_flight, len(valid))
        oldest = None
        if len(valid):
            keys = [(int(lk[t, p, 3]), int(lk[t, p, 1]), t, p) for t, p in valid]
            inj, src, t, p = min(keys)
            at = t + nbr[p]
            dst = int(lk[t, p, 2])
            oldest = (inj, src, at, dst)
        s.step(1)
        if oldest is None:
            continue
        inj, src, at, dst = oldest
        lk2 = s.links()
        hit = [(t, p) for t, p in np.argwhere(lk2[:, :, 0] != 0)
               if int(lk2[t, p, 3]) == inj and int(lk2[t, p, 1]) == src]
        if at == dst:
            assert not hit                                          # ejected
            continue
        assert len(hit) == 1
        t, p = hit[0]
        d0 = abs(at % W - dst % W) + abs(at // W - dst // W)
        nxt = t + nbr[p]
        d1 = abs(nxt % W - dst % W) + abs(nxt // W - dst // W)
        assert d1 == d0 - 1                                          # productive
    st = s.stats()
    assert st["deflections"] > 0
    # age priority bound: latency <= (flits older at injection + 1) * diameter
    assert st["lat_max"] <= (max_in_flight + 1) * (W + H - 2)


def test_mean_distance_closed_form(oracle_mod):
    """In a mesh every productive hop shortens the Manhattan distance by one and
    every deflected hop lengthens it by one, so the summed latency of all
    flits is sum(|dx|+|dy|) + 2 * deflections.  The distance of uniform pairs
    (src != dst) on a WxW mesh has mean 2(W^2-1)/(3W) * N/(N-1)."""
    W = 8
    s = oracle_mod.OracleSim(net_params(W, W, period=400, seed=11))
    s.step(60_000)
    s.drain(10_000)
    st = s.stats()
    n = st["ejected"]
    assert n == st["injected"] > 9000
    N = W * W
    mean = 2 * (W * W - 1) / (3 * W) * N / (N - 1)
    var_axis = (W * W - 1) / 6 - ((W * W - 1) / (3 * W)) ** 2
    sd = np.sqrt(2 * var_axis)
    hops = (st["lat_sum"] - 2 * st["deflections"]) / n
    assert abs(hops - mean) < 5 * sd / np.sqrt(n)


# --------------------------------------------------------------------------
# caches: LRU brute force against an independent OrderedDict model
def lru_model(refs, l1_sets, l1_ways, l2_sets, l2_ways):
    l1 = [OrderedDict() for _ in range(l1_sets)]
    l2 = [OrderedDict() for _ in range(l2_sets)]
    c = Counter()

    def wt(line):
        s2 = l2[line % l2_sets]
        if line in s2:
            s2[line] = 1
            s2.move_to_end(line)
            c["wt_hit"] += 1
        else:
            c["mem_write"] += 1

    for line, write in refs:
        s1 = l1[line % l1_sets]
        if line in s1:
            c["l1_hit"] += 1
            if write:
                wt(line)
            s1.move_to_end(line)
            continue
        c["l1_miss"] += 1
        s2 = l2[line % l2_sets]
        if line in s2:
            c["l2_hit"] += 1
            s2.move_to_end(line)
        else:
            c["l2_miss"] += 1
            if len(s2) == l2_ways:
                _, dirty = s2.popitem(last=False)
                c["mem_wb"] += dirty
            s2[line] = 0
        if len(s1) == l1_ways:
            s1.popitem(last=False)
        s1[line] = 1
        if write:
            wt(line)
    return c


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lru_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    cache = I.cache_cfg()
    cache.update(l1_sets=2, l1_ways=2, l2_sets=4, l2_ways=3)
    p = trace_params(1, 1, period=200, cache=cache)
    lines = rng.integers(0, 40, size=400)
    writes = rng.random(400) < 0.3
    refs = [(int(a), bool(b)) for a, b in zip(lines, writes)]
    s = oracle_mod.OracleSim(p)
    s.set_trace(0, [a | (int(b) << 31) for a, b in refs])
    s.step(400 * 200 + 200)
    st = s.stats()
    want = lru_model(refs, 2, 2, 4, 3)
    for k in ("l1_hit", "l1_miss", "l2_hit", "l2_miss", "wt_hit", "mem_write", "mem_wb"):
        assert st[k] == want[k], k
    assert st["l1_hit"] + st["l1_miss"] == 400
    assert st["injected"] == 0


# --------------------------------------------------------------------------
# hand-worked protocol timelines (interleaved L2), 3x3 mesh, trace input
def test_remote_read_timeline(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3))
    s.set_trace(0, [8])            # line 8: home 8 = (2,2), 4 hops from tile 0
    s.step(112)                                          # cycles 0..111
    assert s.core(0)["om_kind"] == 2                    # still waiting for data
    s.step(1)                                            # cycle 112: DATA ejected
    st = s.stats()
    assert s.core(0)["om_kind"] == 0
    # t=0 L1 miss; t=4 REQ injected; t=8 at home, memory until 108;
    # DATA injected at 108, ejected at tile 0 at 112
    assert st["l2lat_sum"] == 112 and st["l2lat_cnt"] == 1
    assert st["lat_sum"] == 8 and st["ejected"] == 2
    for k in ("req_made", "req_rcvd", "reply_sent", "reply_rcvd", "mem_req", "l1_miss",
              "l2_miss"):
        assert st[k] == 1, k
    l1 = s.cache(0, 1)
    assert (l1[:, :, 0] == 1).sum() == 1 and l1[8 % l1.shape[0], 0, 2] == 8  # owner 8


def test_write_through_timeline(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3))
    s.set_trace(0, [8, 8 | (1 << 31)])
    s.step(203)
    assert s.stats()["wt_sent"] == 1 and s.stats()["wt_hit"] == 0
    s.step(2)                                            # WT ejected at home at 204
    st = s.stats()
    assert st["l1_hit"] == 1 and st["wt_hit"] == 1
    l2 = s.cache(8, 2)
    assert l2[0, 0, 0] == 1 and l2[0, 0, 1] == 8 and (l2[0, 0, 2] & 1) == 1  # dirty


def test_local_home_no_flits(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3))
    s.set_trace(4, [13])           # 13 mod 9 = 4: the home is the requester
    s.step(300)
    st = s.stats()
    assert st["injected"] == 0 and st["l2lat_sum"] == 104 and st["mem_req"] == 1


def test_miss_under_miss_stalls(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3, period=10))
    s.set_trace(0, [8, 17])        # both homed at tile 8
    s.step(400)
    st = s.stats()
    assert st["mm_stall"] == 1 and st["l1_miss"] == 3
    # second reference re-runs at 113: L1 miss, REQ at 117, DATA back at 225
    assert st["l2lat_sum"] == 112 + 112 and st["l2lat_cnt"] == 2


# --------------------------------------------------------------------------
# LSPD directory timelines (Sec. 3.2, Sec. 6.2.2 access sequence)
def test_lspd_negative_then_positive(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3, policy=I.POLICY_LSPD_LOCAL))
    s.set_trace(0, [8])
    s.set_trace(2, [20, 8])        # 20 mod 9 = 2: local directory; then line 8
    s.step(114)
    st = s.stats()
    # DA at 4 -> home at 8 -> DR_NEG injected 9, back at 13 -> memory until 113
    assert s.dir_get(8) == (0 | (1 << 16))
    assert st["l2lat_sum"] == 113 + 104
    l2 = s.cache(0, 2)
    assert any(l2[8 % l2.shape[0], w, 1] == 8 and l2[8 % l2.shape[0], w, 0] for w in range(l2.shape[1]))
    s.step(200)
    st = s.stats()
    # core 2 at 200: DA at 204 -> home 206 -> DR_POS 207 -> back 209 ->
    # REQ injected 210 -> owner 212 -> DATA 213 -> back 215
    assert st["l2lat_sum"] == 113 + 104 + 15
    assert st["req_made"] == 1 and st["req_rcvd"] == 1
    assert st["reply_sent"] == 3 and st["reply_rcvd"] == 3
    assert st["dir_search"] == 3 and st["mem_req"] == 2 and st["trap"] == 0


def test_migration_and_directory_update(oracle_mod):
    cache = I.cache_cfg()
    cache.update(l1_sets=1, l1_ways=1, l2_sets=4, l2_ways=2, mig_window=4, mig_threshold=3)
    s = oracle_mod.OracleSim(trace_params(3, 3, policy=I.POLICY_LSPD_MIGRATE, cache=cache))
    s.set_trace(0, [8])
    s.set_trace(2, [20, 8, 20, 8, 20, 8, 20, 8, 20, 8, 20])
    s.step(2400)
    s.drain(5000)
    st = s.stats()
    assert st["mig_sent"] == 1 and st["migrations"] == 1
    assert s.dir_get(8) & 0xFFFF == 2
    l2_0, l2_2 = s.cache(0, 2), s.cache(2, 2)
    assert not any(l2_0[0, w, 0] and l2_0[0, w, 1] == 8 for w in range(2))
    assert any(l2_2[0, w, 0] and l2_2[0, w, 1] == 8 for w in range(2))
    # the fifth access by core 2 hits its own slice
    assert st["req_made"] == 4
    assert s.core(0)["fwd_n"] == 1


# --------------------------------------------------------------------------
# protocol invariants after a drain (Table 3: requests made == received,
# replies sent == received) on random traffic under every policy
@pytest.mark.parametrize("policy", [0, 1, 2])
def test_table3_conservation_after_drain(oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    p = I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9)
    s = oracle_mod.OracleSim(p)
    s.step(4000)
    s.drain(100_000)
    st = s.stats()
    assert st["injected"] == st["ejected"]
    assert st["req_made"] == st["req_rcvd"] > 0
    assert st["reply_sent"] == st["reply_rcvd"] > 0
    assert st["l2lat_cnt"] == st["l1_miss"] - st["mm_stall"]
    if policy == 2:
        assert st["migrations"] > 0 and st["redir"] + st["trap"] > 0
    if policy == 1:
        # single copy: a line is in at most one slice, and every copy is the
        # one its home's directory names
        where = {}
        for t in range(36):
            l2 = s.cache(t, 2)
            for set_ in range(l2.shape[0]):
                for w in range(l2.shape[1]):
                    if l2[set_, w, 0]:
                        line = int(l2[set_, w, 1])
                        assert line not in where
                        where[line] = t
                        d = s.dir_get(line)
                        assert d & 0xFFFF == t and d >> 16 == l2[set_, w, 2] >> 16


def test_drain_is_a_fixed_point(oracle_mod):
    s = oracle_mod.OracleSim(I.sim_params(4, 4, seed=3, traf=I.traffic(period=5)))
    s.step(1500)
    s.drain(100_000)
    h0, c0 = s.dyn_hash(), s.cycle
    s.step(50)
    assert s.dyn_hash() == h0 and s.cycle == c0 + 50


def test_hash_trace_is_deterministic_and_seeded(oracle_mod):
    a = oracle_mod.OracleSim(I.MESH_8["params"]).step(300, trace=True)
    b = oracle_mod.OracleSim(I.MESH_8["params"]).step(300, trace=True)
    p = dict(I.MESH_8["params"], seed=2)
    c = oracle_mod.OracleSim(p).step(300, trace=True)
    assert (a == b).all() and (a != c).any()


def test_service_queue_overflow_is_an_error(oracle_mod):
    p = I.sim_params(8, 8, seed=1, cache=I.cache_cfg(svc_q=1),
                     traf=I.traffic(period=1, priv=0.0, shared=1.0, hot=1.0, hot_side=1,
                                    shared_mb=1))
    s = oracle_mod.OracleSim(p)
    rc = s.step(20_000, check=False)
    code, cyc = s.error()
    assert rc == 3 and code == 3 and cyc > 0
    s2 = oracle_mod.OracleSim(p)
    s2.step(20_000, check=False)
    assert s2.error() == (code, cyc)


# --------------------------------------------------------------------------
# the reference stream: region fractions, bounds, write fraction, hotspot
def test_reference_stream_distribution(oracle_mod):
    p = I.mesh_64(1)
    s = oracle_mod.OracleSim(p)
    N = 64 * 64
    rb, sb = p["remote_lines"], p["remote_lines"] + p["shared_lines"]
    cnt = Counter()
    hot_tiles = {y * 64 + x for x in range(30, 34) for y in range(30, 34)}
    hot = shared = 0
    n = 120_000
    for i in range(n):
        core, k = i % N, i // N
        line, w = s.draw_ref(core, k)
        cnt["w"] += w
        if line < rb:
            cnt["remote"] += 1
        elif line < sb:
            cnt["shared"] += 1
            shared += 1
            hot += (line % N) in hot_tiles
        else:
            cnt["priv"] += 1
            base = sb + core * p["priv_lines"]
            assert base <= line < base + p["priv_lines"]
    for k, f in (("priv", 0.7), ("shared", 0.2), ("remote", 0.1), ("w", 0.3)):
        sd = np.sqrt(f * (1 - f) / n)
        assert abs(cnt[k] / n - f) < 5 * sd, k
    f_hot = 0.4 + 0.6 * 16 / N
    sd = np.sqrt(f_hot * (1 - f_hot) / shared)
    assert abs(hot / shared - f_hot) < 5 * sd


def test_hotspot_lines_exactly_the_hot_tiles_shared_lines(oracle_mod):
    """Every shared reference sent to the hot block (hot fraction 1) is a line
    of the shared region homed (line mod N) on one of the 4x4 centre tiles
    x, y in [W/2-2, W/2+1]; over enough draws the lines drawn are exactly those
    lines, each about equally often; with hot fraction 0 they are exactly
    the whole shared region.  Checked per draw against the definition of the
    region and of the home, not against the mapping's own arithmetic."""
    W = H = 8
    N = W * H
    traf = I.traffic(period=1, priv=0.0, shared=1.0, hot=1.0, hot_side=4, shared_mb=0)
    traf.update(shared_lines=640)
    p = I.sim_params(W, H, traf=traf, seed=3)
    sb = p["remote_lines"]
    hot_tiles = {y * W + x for x in range(W // 2 - 2, W // 2 + 2) for y in range(H // 2 - 2, H // 2 + 2)}
    want = {l for l in range(sb, sb + 640) if l % N in hot_tiles}
    assert len(want) == 160
    s = oracle_mod.OracleSim(p)
    seen = Counter()
    for i in range(24_000):
        line, _ = s.draw_ref(i % N, i // N)
        assert line in want, line
        seen[line] += 1
    assert set(seen) == want
    # uniform over the 160 lines: chi-square with 159 degrees of freedom
    e = 24_000 / 160
    chi2 = sum((v - e) ** 2 / e for v in seen.values())
    assert chi2 < 159 + 6 * np.sqrt(2 * 159)
    s.close()
    p0 = dict(p, hot_q16=0)
    s = oracle_mod.OracleSim(p0)
    lines = {s.draw_ref(i % N, i // N)[0] for i in range(20_000)}
    assert lines == set(range(sb, sb + 640))
    s.close()


# --------------------------------------------------------------------------
# packet mode (Table 1): a data reply is 4 flits, reassembled in a reorder
# buffer; its handler runs once, when the last flit is in
def test_packet_remote_read_timeline(oracle_mod):
    s = oracle_mod.OracleSim(trace_params(3, 3, packet_mode=1, rob_entries=4))
    s.set_trace(0, [8])            # as the one-flit timeline: home 8, 4 hops
    s.step(113)                                          # cycles 0..112
    assert s.core(0)["om_kind"] == 2          # first flit in at 112, three to go
    s.step(2)                                            # cycles 113, 114
    assert s.core(0)["om_kind"] == 2
    s.step(1)                                            # cycle 115: the 4th flit
    st = s.stats()
    assert s.core(0)["om_kind"] == 0
    # the four flits leave home at 108..111 and arrive at 112..115
    assert st["l2lat_sum"] == 115 and st["l2lat_cnt"] == 1
    assert st["injected"] == st["ejected"] == 5
    assert st["lat_sum"] == 4 + 4 * 4
    assert st["reply_sent"] == st["reply_rcvd"] == 1


def test_packet_handler_runs_on_the_last_flit_in_any_order(oracle_mod):
    s = oracle_mod.OracleSim(quiet_params(3, 3, packet_mode=1, rob_entries=4))
    s.step(10)
    h = s.dyn_hash()
    for k, idx in enumerate((2, 0, 3, 1)):       # out of order, one per cycle
        s.debug_link(4, W_, dict(type="DATA", src=3, dst=4, inject=9 + k, line=11, a=idx, e=4))
        s.step(1, check=False)
        if k < 3:
            assert s.error()[0] == 0
            assert s.dyn_hash() != h             # the partial packet is state
            h = s.dyn_hash()
    # no miss is outstanding at tile 4, so the completed reply is a protocol
    # error -- raised exactly at the cycle the fourth flit was ejected
    assert s.error() == (6, 13)
    assert s.stats()["reply_rcvd"] == 1


def test_packet_reorder_buffer_overflow(oracle_mod):
    s = oracle_mod.OracleSim(quiet_params(3, 3, packet_mode=1, rob_entries=1))
    s.step(10)
    s.debug_link(4, W_, dict(type="DATA", src=3, dst=4, inject=5, line=11, a=0, e=4))
    s.debug_link(4, N_, dict(type="DATA", src=1, dst=4, inject=7, line=13, a=0, e=4))
    s.step(5, check=False)
    # the older flit takes the only entry at cycle 10; the younger, deflected
    # north and back, needs a second entry when it is ejected at cycle 12
    assert s.error() == (3, 12)


def test_packet_mode_conservation_after_drain(oracle_mod):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, svc_q=512, packet_mode=1,
                        rob_entries=8)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    s = oracle_mod.OracleSim(I.sim_params(6, 6, policy=0, cache=cache, traf=traf, seed=9))
    s.step(4000)
    s.drain(100_000)
    st = s.stats()
    assert st["injected"] == st["ejected"]
    assert st["req_made"] == st["req_rcvd"] > 0
    assert st["reply_sent"] == st["reply_rcvd"] > 0
    # interleaved L2: requests and write-throughs are one flit, every reply a
    # 4-flit data packet
    assert st["injected"] == st["req_made"] + st["wt_sent"] + 4 * st["reply_sent"]


# --------------------------------------------------------------------------
# centralized directory node (Sec. 3.2's alternative): every directory message
# goes to one tile instead of the line's home
def test_central_directory_timeline(oracle_mod):
    dist = oracle_mod.OracleSim(trace_params(3, 3, policy=I.POLICY_LSPD_LOCAL))
    cent = oracle_mod.OracleSim(trace_params(3, 3, policy=I.POLICY_LSPD_LOCAL, dir_central=1,
                                             dir_tile=1))
    for s in (dist, cent):
        s.set_trace(0, [8])        # home 8 is 4 hops from tile 0; tile 1 is 1 hop
        s.step(150)
    a, b = dist.stats(), cent.stats()
    # DA out and DR_NEG back each travel 3 hops fewer
    assert a["l2lat_sum"] == 113 and b["l2lat_sum"] == 113 - 2 * 3
    assert a["dir_search"] == b["dir_search"] == 1
    assert cent.stats(1)["dir_search"] == 1 and dist.stats(8)["dir_search"] == 1
    assert cent.dir_get(8) == dist.dir_get(8) == (0 | (1 << 16))


@pytest.mark.parametrize("policy", [1, 2])
def test_central_directory_takes_every_lookup(oracle_mod, policy):
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, dir_central=1, dir_tile=14)
    traf = I.traffic(period=3, write=0.3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=300)
    s = oracle_mod.OracleSim(I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=9))
    s.step(4000)
    s.drain(100_000)
    st = s.stats()
    assert st["dir_search"] > 0 and s.stats(14)["dir_search"] == st["dir_search"]
    assert st["injected"] == st["ejected"]
    assert st["req_made"] == st["req_rcvd"] and st["reply_sent"] == st["reply_rcvd"]
    if policy == 2:
        assert st["migrations"] > 0 and s.stats(14)["migrations"] == st["migrations"]


# --------------------------------------------------------------------------
# L1 write-back option: a write dirties the L1 copy; a dirty victim is written
# to the L2 that supplied it (local slice, another tile, or memory)
def lru_model_write_back(refs, l1_sets, l1_ways, l2_sets, l2_ways):
    l1 = [OrderedDict() for _ in range(l1_sets)]      # line -> dirty
    l2 = [OrderedDict() for _ in range(l2_sets)]
    c = Counter()

    def to_l2(line):
        s2 = l2[line % l2_sets]
        if line in s2:
            s2[line] = 1
            s2.move_to_end(line)
            c["wt_hit"] += 1
        else:
            c["mem_write"] += 1

    for line, write in refs:
        s1 = l1[line % l1_sets]
        if line in s1:
            c["l1_hit"] += 1
            if write:
                s1[line] = 1
            s1.move_to_end(line)
            continue
        c["l1_miss"] += 1
        s2 = l2[line % l2_sets]
        if line in s2:
            c["l2_hit"] += 1
            s2.move_to_end(line)
        else:
            c["l2_miss"] += 1
            if len(s2) == l2_ways:
                _, dirty = s2.popitem(last=False)
                c["mem_wb"] += dirty
            s2[line] = 0
        if len(s1) == l1_ways:
            victim, vdirty = s1.popitem(last=False)
            if vdirty:
                to_l2(victim)
        s1[line] = 1 if write else 0
    return c


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_l1_write_back_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    cache = I.cache_cfg(l1_write_back=1)
    cache.update(l1_sets=2, l1_ways=2, l2_sets=4, l2_ways=3)
    p = trace_params(1, 1, period=200, cache=cache)
    lines = rng.integers(0, 40, size=400)
    writes = rng.random(400) < 0.3
    refs = [(int(a), bool(b)) for a, b in zip(lines, writes)]
    s = oracle_mod.OracleSim(p)
    s.set_trace(0, [a | (int(b) << 31) for a, b in refs])
    s.step(400 * 200 + 200)
    st = s.stats()
    want = lru_model_write_back(refs, 2, 2, 4, 3)
    for k in ("l1_hit", "l1_miss", "l2_hit", "l2_miss", "wt_hit", "mem_write", "mem_wb"):
        assert st[k] == want[k], k
    # write-back generates fewer L2 writes than write-through on the same refs
    wt = lru_model(refs, 2, 2, 4, 3)
    assert want["wt_hit"] + want["mem_write"] <= wt["wt_hit"] + wt["mem_write"]


def test_l1_write_back_timeline(oracle_mod):
    # core 0 reads line 8 (home 8, remote), writes it (an L1 hit), then four
    # more lines of the same L1 set evict it: only then does a WT go home
    l1_sets = I.cache_cfg()["l1_sets"]
    refs = [8, 8 | (1 << 31)] + [8 + k * l1_sets for k in range(1, 5)]
    s = oracle_mod.OracleSim(trace_params(3, 3, l1_write_back=1))
    s.set_trace(0, refs)
    s.step(2 * 200 + 50)
    assert s.stats()["wt_sent"] == 0 and s.stats()["l1_hit"] == 1
    s.step(6 * 200)
    st = s.stats()
    assert st["wt_sent"] == 1 and st["wt_hit"] == 1 and st["l1_miss"] == 5
    l2 = s.cache(8, 2)
    assert any(l2[0, w, 0] and l2[0, w, 1] == 8 and (l2[0, w, 2] & 1) for w in range(l2.shape[1]))
    wt = oracle_mod.OracleSim(trace_params(3, 3))
    wt.set_trace(0, refs)
    wt.step(2 * 200 + 50)
    assert wt.stats()["wt_sent"] == 1                  # write-through: at the write


# --------------------------------------------------------------------------
# age_mode 1: the paper's age field, a count of deflections (Sec. 4.2, 6.2.1,
# 7.1) -- most deflections first, ties by inject cycle, then source tile
def one_router_model(arrivals, queued, here, W, H, t, age_mode):
    """An independent model of one router's cycle (Sec. 4.3): arrivals is a
    list of (input port, flit dict); returns (ejected flit, {out port: flit},
    deflections).  Written from the rules, not from either simulator."""
    x, y = here % W, here // W
    exists = [y > 0, y < H - 1, x < W - 1, x > 0]           # N, S, E, W
    def key(f):
        return ((-f["age"] if age_mode else 0), f["inject"], f["src"])
    flits = [dict(f) for _, f in arrivals]
    mine = [f for f in flits if f["dst"] == here]
    ej = min(mine, key=key) if mine else None
    rest = sorted((f for f in flits if f is not ej), key=key)
    if len(arrivals) < sum(exists) and queued is not None:
        rest.append(dict(queued, inject=t, src=here, age=0))
    out, defl = {}, 0
    for f in rest:
        dx, dy = f["dst"] % W - x, f["dst"] // W - y
        xp = E_ if dx > 0 else (W_ if dx < 0 else None)
        yp = S_ if dy > 0 else (N_ if dy < 0 else None)
        port = next(p for p in (xp, yp, N_, S_, E_, W_)
                    if p is not None and exists[p] and p not in out)
        if port not in (xp, yp):
            defl += 1
            if age_mode:
                f["age"] += 1
        out[port] = f
    return ej, out, defl


@pytest.mark.parametrize("age_mode", [0, 1])
@pytest.mark.parametrize("here", [4, 1, 0])
def test_one_router_brute_force(oracle_mod, age_mode, here):
    W = H = 3
    rng = np.random.default_rng(100 + 10 * here + age_mode)
    x, y = here % W, here // W
    ports = [p for p, ok in zip((N_, S_, E_, W_), (y > 0, y < H - 1, x < W - 1, x > 0)) if ok]
    for trial in range(120):
        s = oracle_mod.OracleSim(quiet_params(W, H, age_mode=age_mode))
        s.step(10)
        k = int(rng.integers(0, len(ports) + 1))
        used = rng.choice(ports, size=k, replace=False)
        srcs = rng.choice([r for r in range(9) if r != here], size=k, replace=False)
        arrivals = []
        for p, src in zip(used, srcs):
            f = dict(type="PROBE", src=int(src), dst=int(rng.integers(0, 9)),
                     inject=int(rng.integers(0, 4)), age=int(rng.integers(0, 3)) if age_mode else 0)
            s.debug_link(here, int(p), f)
            arrivals.append((int(p), f))
        queued = None
        if rng.random() < 0.6:
            queued = dict(type="PROBE", dst=int(rng.choice([r for r in range(9) if r != here])))
            s.debug_enqueue(here, 0, queued)
        ej, out, defl = one_router_model(arrivals, queued, here, W, H, 10, age_mode)
        s.step(1)
        st = s.stats()
        assert st["deflections"] == defl, trial
        assert st["ejected"] == (1 if ej else 0), trial
        if ej:
            assert st["lat_sum"] == 10 - ej["inject"], trial
        lk = s.links()[here]
        for p in range(4):
            if p in out:
                f = out[p]
                assert (lk[p, 1], lk[p, 2], lk[p, 3], lk[p, 7]) == \
                    (f["src"], f["dst"], f["inject"], f["age"]), (trial, p)
            else:
                assert lk[p, 0] == 0, (trial, p)


def test_deflection_age_conflict(oracle_mod):
    """The conflict of test_two_flit_conflict under age_mode 1: the younger
    flit B has been deflected twice, so it takes port E and the older A is
    deflected north and ages by one; with equal ages the older one wins."""
    s = oracle_mod.OracleSim(quiet_params(3, 3, age_mode=1))
    s.step(10)
    s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=0))
    s.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=7, age=2))
    s.step(1)
    lk = s.links()
    assert lk[4, E_][1] == 1 and lk[4, E_][7] == 2
    assert lk[4, N_][1] == 3 and lk[4, N_][7] == 1
    s.step(5)
    st = s.stats()
    # B: one hop (cycle 11); A: N, then E, then S (cycle 13)
    assert st["ejected"] == 2 and st["lat_sum"] == (11 - 7) + (13 - 5)
    t = oracle_mod.OracleSim(quiet_params(3, 3, age_mode=1))
    t.step(10)
    t.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=1))
    t.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=7, age=1))
    t.step(1)
    lk = t.links()
    assert lk[4, E_][1] == 3 and lk[4, N_][1] == 1 and lk[4, N_][7] == 2
    # age_mode 0 ignores the age field: a planted age is refused there
    u = oracle_mod.OracleSim(quiet_params(3, 3))
    with pytest.raises(ValueError):
        u.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=1))


def test_deflection_age_top_flit_never_deflected(oracle_mod):
    """Under load with age_mode 1 the flit of highest priority in the whole
    network (most deflections, then oldest, then lowest source) is never
    deflected: it ejects or moves one hop closer every cycle; flits do age."""
    W = H = 6
    p = net_params(W, H, period=2)
    p["age_mode"] = 1
    s = oracle_mod.OracleSim(p)
    nbr = {N_: -W, S_: W, E_: 1, W_: -1}
    top_age = 0
    for _ in range(400):
        lk = s.links()
        valid = np.argwhere(lk[:, :, 0] != 0)
        st = s.stats()
        assert len(valid) == st["injected"] - st["ejected"]
        if not len(valid):
            s.step(1)
            continue
        keys = [(-int(lk[t, p, 7]), int(lk[t, p, 3]), int(lk[t, p, 1]), t, p) for t, p in valid]
        nage, inj, src, t, p = min(keys)
        top_age = max(top_age, -nage)
        at, dst = t + nbr[p], int(lk[t, p, 2])
        s.step(1)
        lk2 = s.links()
        hit = [(t2, p2) for t2, p2 in np.argwhere(lk2[:, :, 0] != 0)
               if int(lk2[t2, p2, 3]) == inj and int(lk2[t2, p2, 1]) == src]
        if at == dst:
            assert not hit
            continue
        assert len(hit) == 1
        t2, p2 = hit[0]
        assert int(lk2[t2, p2, 7]) == -nage                          # not aged
        d0 = abs(at % W - dst % W) + abs(at // W - dst // W)
        nxt = t2 + nbr[p2]
        assert abs(nxt % W - dst % W) + abs(nxt // W - dst // W) == d0 - 1
    assert top_age >= 2 and s.stats()["deflections"] > 0


def test_deflection_age_limits(oracle_mod):
    """age_mode 1 counts at most 4095 deflections per flit (one more is error
    8 in that cycle) and runs at most 2^20 cycles (a longer step or drain is
    refused as an argument error before it runs)."""
    s = oracle_mod.OracleSim(quiet_params(3, 3, age_mode=1))
    s.step(10)
    s.debug_link(4, W_, dict(type="PROBE", src=3, dst=5, inject=5, age=4095))
    s.debug_link(4, N_, dict(type="PROBE", src=1, dst=5, inject=7, age=4095))
    assert s.step(1, check=False) == 8
    assert s.error() == (8, 10)
    t = oracle_mod.OracleSim(quiet_params(3, 3, age_mode=1))
    assert t.step((1 << 20) + 1, check=False) == 1 and t.cycle == 0
    with pytest.raises(Exception):
        t.drain((1 << 20) + 1)
    t.step(1000)
    assert t.step((1 << 20) - 999, check=False) == 1 and t.cycle == 1000
    u = oracle_mod.OracleSim(quiet_params(3, 3))                   # age_mode 0: no limit
    assert u.step((1 << 20) + 1, check=False) == 0


def test_full_length_records_match_the_oracle_now(oracle_mod):
    """The stored full-length records (tests/golden/full_length.json) are the
    oracle's: the first checkpoint of a 64x64 run and of a 208x208 run,
    recomputed now, equals the stored one (so a change to the oracle or to the
    workload parameters cannot leave the GPU tests comparing against stale
    values)."""
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_length.json")
    with open(path) as fh:
        wl = json.load(fh)["workloads"]
    from paper_1508_03235_b300 import inputs as I
    assert wl["mesh64_hotspot_seed1"]["params"] == I.mesh_64(1)
    assert wl["mesh208_period40"]["params"] == I.mesh_208(40)
    for name in ("mesh64_hotspot_seed1", "mesh208_period40"):
        rec = wl[name]["checkpoints"][0]
        o = oracle_mod.OracleSim(wl[name]["params"])
        o.step(rec["cycle"])
        assert o.stats() == rec["stats"], name
        assert str(o.dyn_hash()) == rec["dyn_hash"] and str(o.state_hash()) == rec["state_hash"]
        assert [{str(i): int(v) for i, v in enumerate(o.hist(w)) if v} for w in (0, 1)] == rec["hist"]
        o.close()


def test_batch_records_match_the_oracle_now(oracle_mod):
    """The stored 512-instance records (tests/golden/batch_c3.json) are the
    oracle's: two small instances recomputed now equal their records."""
    import hashlib
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_c3.json")
    with open(path) as fh:
        doc = json.load(fh)
    pts = I.batch_design_points(doc["instances"], seed=doc["design_seed"])
    small = sorted(range(len(pts)), key=lambda i: (pts[i]["mesh_w"], i))[:2]
    for i in small:
        p = dict(pts[i])
        p.pop("design")
        o = oracle_mod.OracleSim(p)
        o.step(doc["cycles"])
        rec = doc["records"][i]
        assert o.stats() == rec["stats"] and str(o.state_hash()) == rec["state_hash"], i
        dig = [hashlib.sha256(np.ascontiguousarray(o.hist(w), dtype="<u8").tobytes()).hexdigest()[:16]
               for w in (0, 1)]
        assert dig == rec["hist_sha"], i
        o.close()
