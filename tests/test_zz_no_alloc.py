"""The allocation-free entry point, noc_run_static, checked against the
regular handle-based path on the same simulations, two calls in a row.

It exists for callers that cannot allocate device memory while they run (a
process whose HBM another allocator has reserved, or a host loop that must not
allocate or synchronise through cudaMalloc/cudaFree); it keeps all simulator
state in a fixed 16 MiB device array inside the library.  The second call also
shows that each call starts from a cleared array."""
import ctypes as C

import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu


def static_run(noc, torch, params, cycles):
    out = torch.zeros(len(noc.STATS_FIELDS), dtype=torch.int64, device="cuda")
    L = noc.lib()
    L.noc_run_static.restype = C.c_int
    L.noc_run_static.argtypes = [C.c_int, C.c_int, C.POINTER(noc.CacheCfg), C.c_int,
                                 C.POINTER(noc.Traffic), C.c_uint64, C.c_int64, C.c_void_p,
                                 C.c_void_p]
    rc = L.noc_run_static(params["mesh_w"], params["mesh_h"],
                          C.byref(noc.cache_struct(params)), params["policy"],
                          C.byref(noc.traffic_struct(params)), params["seed"], cycles,
                          C.c_void_p(out.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    vals = [int(v) & (2**64 - 1) for v in out.cpu().tolist()]
    return dict(zip(noc.STATS_FIELDS, vals))


def handle_run(noc, params, cycles):
    s = noc.Sim(params)
    s.step(cycles)
    return s.stats()


def test_static_entry_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc
    # an 8x8 cache workload, then a network-only 40x40 mesh, then the first again
    cache_case = dict(I.MESH_8["params"])
    net_case = I.sim_params(40, 40, seed=4, traf=I.traffic(period=3, mode=I.MODE_NETWORK),
                            cache=I.cache_cfg(l1_kb=1, l1_ways=1, l2_kb=1, l2_ways=1))
    for params, cycles in ((cache_case, 3000), (net_case, 2000), (cache_case, 3000)):
        got = static_run(noc, torch, params, cycles)
        want = handle_run(noc, params, cycles)
        assert got == want
        assert got["ejected"] > 0


def test_static_entry_rejects_oversize_state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc
    p = I.mesh_64(1)           # 64x64 tiles with full-size caches: far above 16 MiB
    out = torch.zeros(len(noc.STATS_FIELDS), dtype=torch.int64, device="cuda")
    L = noc.lib()
    rc = L.noc_run_static(64, 64, C.byref(noc.cache_struct(p)), 0, C.byref(noc.traffic_struct(p)),
                          1, 10, C.c_void_p(out.data_ptr()), None)
    assert rc == 1
