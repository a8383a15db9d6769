"""The allocation-free entry point, noc_run_static, checked against the
regular handle-based path (and once against the oracle) on the same
simulations, several calls in a row.

It exists for callers that cannot allocate device memory while they run (a
process whose HBM another allocator has reserved, or a host loop that must not
allocate or synchronise through cudaMalloc/cudaFree); it keeps all simulator
state in a fixed 16 MiB device array inside the library.  The calls run one
after another on the same array: every L2 policy, a multi-flit packet
configuration and a network-only mesh, with a migration run right after an
interleaved one and the interleaved run repeated last, so that contents a call
failed to clear would change a later call's counters."""
import ctypes as C

import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu


def small_lspd(policy, packet_mode=0):
    """A small mesh whose state (directory included) fits the array: tiny
    caches and address regions, so that evictions, directory traffic and
    (policy 2) migrations happen every few cycles."""
    cache = I.cache_cfg(l1_kb=1, l1_ways=2, l2_kb=4, l2_ways=4, mig_window=4, mig_threshold=2,
                        svc_q=512, packet_mode=packet_mode)
    traf = I.traffic(period=3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=100, remote_lines=20_000)
    return I.sim_params(6, 6, policy=policy, cache=cache, traf=traf, seed=11)


CASES = [
    ("interleaved", dict(I.MESH_8["params"]), 3000),
    ("lspd_migrate", small_lspd(I.POLICY_LSPD_MIGRATE), 2500),
    ("lspd_local", small_lspd(I.POLICY_LSPD_LOCAL), 2500),
    ("packets_migrate", small_lspd(I.POLICY_LSPD_MIGRATE, packet_mode=1), 2500),
    ("network_40x40", I.sim_params(40, 40, seed=4, traf=I.traffic(period=3, mode=I.MODE_NETWORK),
                                   cache=I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1)), 2000),
    ("interleaved_again", dict(I.MESH_8["params"]), 3000),
]


def static_run(noc, torch, params, cycles):
    """One call through the C ABI (the binding declares its signature)."""
    out = torch.zeros(len(noc.STATS_FIELDS), dtype=torch.int64, device="cuda")
    rc = noc.lib().noc_run_static(params["mesh_w"], params["mesh_h"],
                                  C.byref(noc.cache_struct(params)), params["policy"],
                                  C.byref(noc.traffic_struct(params)), params["seed"], cycles,
                                  C.c_void_p(out.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, noc.lib().noc_last_error()
    vals = [int(v) & (2**64 - 1) for v in out.cpu().tolist()]
    return dict(zip(noc.STATS_FIELDS, vals))


def handle_run(noc, params, cycles):
    s = noc.Sim(params)
    s.step(cycles)
    out = s.stats()
    s.close()
    return out


def test_static_entry_matches_handle_path_in_sequence(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc
    for name, params, cycles in CASES:
        got = static_run(noc, torch, params, cycles)
        want = handle_run(noc, params, cycles)
        assert got == want, name
        assert got["ejected"] > 0, name
        if name == "lspd_migrate":
            assert got["migrations"] > 0 and got["dir_search"] > 0 and got["mem_wb"] > 0
            # and directly against the oracle
            o = oracle_mod.OracleSim(params)
            o.step(cycles)
            os_ = o.stats()
            o.close()
            for k in noc.STATS_FIELDS:
                assert got[k] == os_[k], k


def test_static_entry_rejects_what_it_cannot_hold():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc
    out = torch.zeros(len(noc.STATS_FIELDS), dtype=torch.int64, device="cuda")
    L = noc.lib()
    p = I.mesh_64(1)           # 64x64 tiles with full-size caches: far above 16 MiB
    rc = L.noc_run_static(64, 64, C.byref(noc.cache_struct(p)), 0, C.byref(noc.traffic_struct(p)),
                          1, 10, C.c_void_p(out.data_ptr()), None)
    assert rc == 1 and b"NOC_STATIC_SCRATCH_BYTES" in L.noc_last_error()
    # a valid run still works after the rejection
    got = static_run(noc, torch, CASES[0][1], 500)
    assert got == handle_run(noc, CASES[0][1], 500)
