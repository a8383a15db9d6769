"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; the binding's structs match the header's layout."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(noc_\w+|mlp_\w+|nocb_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libnoc():
    from paper_1508_03235_b300 import build
    build.build()
    return C.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(libnoc):
    names = declared()
    assert "noc_create" in names and "noc_step" in names and "noc_stats" in names
    missing = [n for n in sorted(names) if not hasattr(libnoc, n)]
    assert not missing, missing


def test_every_kernel_build_the_dispatcher_names_is_linked(libnoc):
    """The library defines a launcher for every build the dispatcher picks --
    each way class x kind x launch bound of the plain loop, the profiled
    builds, the batch kernels -- and leaves no internal symbol undefined."""
    import shutil
    import subprocess
    from paper_1508_03235_b300 import build
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    out = subprocess.run(["nm", "-D", "-C", build.LIB], capture_output=True, text=True, check=True).stdout
    assert not [l for l in out.splitlines() if " U " in l and "noc::" in l]
    defined = {m.group(1) for m in re.finditer(r" T (noc::\w+)\(", out)}
    classes = ("4_8", "4_16", "16_16")
    kinds = ("gen", "base", "il", "local", "migrate")
    want = {f"noc::launch_run_0_0_{c}_{k}{s}" for c in classes for k in kinds for s in ("", "_narrow", "_xl")}
    want |= {f"noc::launch_run_0_0_{c}_{k}_prof" for c in classes for k in ("gen", "base", "il")}
    want |= {f"noc::launch_run_0_0_{c}_gen_checked" for c in classes}
    want |= {f"noc::launch_run_{h}_{c}_gen" for c in classes for h in ("1_0", "0_1")}
    want |= {f"noc::launch_batch_{c}_{k}" for c in classes for k in kinds}
    want |= {f"noc::launch_multi_{c}" for c in classes}
    assert not sorted(want - defined), sorted(want - defined)[:10]


def test_struct_layouts_match_header(libnoc):
    from paper_1508_03235_b300 import noc
    assert C.sizeof(noc.CacheCfg) == 18 * 4
    assert C.sizeof(noc.Traffic) == 11 * 4
    assert C.sizeof(noc.Stats) == 30 * 8
    hdr = open(os.path.join(ROOT, "include", "noc.h")).read()
    body = hdr[hdr.index("typedef struct {\n  uint64_t cycle;"):]
    body = body[:body.index("} noc_stats_t;")]
    fields = re.findall(r"(\w+)[,;]", body.replace("uint64_t", ""))
    assert tuple(fields) == noc.STATS_FIELDS


def test_no_gpu_calls_fail_cleanly_without_device(libnoc):
    """create/required_bytes/destroy are host-only and work on a CPU machine."""
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc
    p = I.MESH_8["params"]
    h = C.c_void_p()
    rc = noc.lib().noc_create(8, 8, C.byref(noc.cache_struct(p)), 0,
                              C.byref(noc.traffic_struct(p)), 1, C.byref(h))
    assert rc == 0
    assert noc.lib().noc_required_bytes(h) > 8 * 8 * 512 * 8 * 4
    bad = noc.cache_struct(dict(p, l1_ways=17))
    h2 = C.c_void_p()
    assert noc.lib().noc_create(8, 8, C.byref(bad), 0, C.byref(noc.traffic_struct(p)), 1,
                                C.byref(h2)) == 1
    assert b"ways" in noc.lib().noc_last_error()
    noc.lib().noc_destroy(h)


def test_stat_names_agree_with_oracle(oracle_mod):
    from paper_1508_03235_b300 import noc
    assert set(oracle_mod.STAT_NAMES) | {"cycle", "in_flight"} == set(noc.STATS_FIELDS)


INVALID = {
    "l2_ways32": dict(l2_ways=32), "l1_sets0": dict(l1_sets=0), "mesh0": dict(mesh_w=0),
    "mesh_too_big": dict(mesh_w=300, mesh_h=300), "policy3": dict(policy=3),
    "mem_latency0": dict(mem_latency=0), "svc_q0": dict(svc_q=0), "core_q0": dict(core_q=0),
    "mem_q0": dict(mem_q=0), "l1_miss_neg": dict(l1_miss_cycles=-1), "packet2": dict(packet_mode=2),
    "rob0": dict(packet_mode=1, rob_entries=0), "rob65": dict(packet_mode=1, rob_entries=65),
    "packets_small_svc_q": dict(packet_mode=1, svc_q=8), "dir_tile_off_mesh": dict(dir_central=1, dir_tile=64),
    "dir2": dict(dir_central=2), "write_back2": dict(l1_write_back=2), "age2": dict(age_mode=2),
    "period_neg": dict(period=-1), "write_frac_big": dict(write_q16=70000),
    "mig_window31": dict(policy=2, mig_window=31), "mig_threshold0": dict(policy=2, mig_threshold=0),
    "fwd0": dict(policy=2, fwd_entries=0), "hot_side_big": dict(hot_side=9), "mode3": dict(mode=3),
    "priv_lines0": dict(priv_lines=0),
}
VALID = {
    "mesh8": {}, "odd_ways": dict(l1_ways=3, l2_ways=6), "ways16": dict(l1_ways=16, l2_ways=16),
    "packets": dict(packet_mode=1), "dir_node": dict(policy=1, dir_central=1, dir_tile=63),
    "every_option": dict(policy=2, packet_mode=1, dir_central=1, dir_tile=5, l1_write_back=1,
                         age_mode=1),
    "window_unused": dict(policy=0, mig_window=31),
}


@pytest.mark.parametrize("name", sorted(INVALID) + sorted(VALID))
def test_library_and_oracle_accept_the_same_configurations(libnoc, oracle_mod, name):
    """noc_create (host-only, no GPU needed) and the oracle agree on which
    configurations are valid; a rejected one is NOC_ERR_ARG with a message."""
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc
    p = dict(I.MESH_8["params"])
    p.update(INVALID.get(name) or VALID.get(name))
    h = C.c_void_p()
    rc = noc.lib().noc_create(p["mesh_w"], p["mesh_h"], C.byref(noc.cache_struct(p)), p["policy"],
                              C.byref(noc.traffic_struct(p)), 1, C.byref(h))
    if rc == 0:
        noc.lib().noc_destroy(h)
    try:
        oracle_mod.OracleSim(p).close()
        oracle_ok = True
    except ValueError:
        oracle_ok = False
    want = name in VALID
    assert (rc == 0) == want and oracle_ok == want, (rc, oracle_ok)
    if not want:
        assert rc == 1 and noc.lib().noc_last_error()


@pytest.mark.parametrize("name", sorted(INVALID) + ["trace_mode", "priv_lines0_cache"])
def test_static_entry_rejects_what_noc_create_rejects(libnoc, name):
    """noc_run_static checks its arguments with noc_create's own checks (plus
    trace mode, which it cannot hold) before any CUDA call, so a rejection
    needs no GPU: NOC_ERR_ARG with a message."""
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc
    p = dict(I.MESH_8["params"])
    p.update(INVALID.get(name) or dict(trace_mode=dict(mode=I.MODE_TRACE),
                                       priv_lines0_cache=dict(priv_lines=0, priv_q16=1000))[name])
    out = (C.c_uint64 * 30)()
    L = noc.lib()
    L.noc_last_error()
    rc = L.noc_run_static(p["mesh_w"], p["mesh_h"], C.byref(noc.cache_struct(p)), p["policy"],
                          C.byref(noc.traffic_struct(p)), 1, 100, C.cast(out, C.c_void_p), None)
    assert rc == 1
    msg = L.noc_last_error()
    assert msg and (name != "trace_mode" or b"trace" in msg)


def test_checkpoint_images_are_checked_before_the_device(libnoc):
    """noc_load rejects what is not an image of this configuration without a
    GPU; the image size is header + arena (host-only)."""
    from paper_1508_03235_b300 import inputs as I
    from paper_1508_03235_b300 import noc
    L = noc.lib()
    p = I.MESH_8["params"]
    h = C.c_void_p()
    assert L.noc_create(8, 8, C.byref(noc.cache_struct(p)), 0, C.byref(noc.traffic_struct(p)), 1,
                        C.byref(h)) == 0
    n = L.noc_checkpoint_bytes(h)
    assert n > L.noc_required_bytes(h)
    junk = (C.c_uint8 * 256)()
    assert L.noc_load(h, C.cast(junk, C.c_void_p), 256) == 1
    assert b"checkpoint" in L.noc_last_error()
    L.noc_destroy(h)
