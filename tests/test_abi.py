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
    bad = noc.cache_struct(dict(p, l1_ways=3))
    h2 = C.c_void_p()
    assert noc.lib().noc_create(8, 8, C.byref(bad), 0, C.byref(noc.traffic_struct(p)), 1,
                                C.byref(h2)) == 1
    assert b"ways" in noc.lib().noc_last_error()
    noc.lib().noc_destroy(h)


def test_stat_names_agree_with_oracle(oracle_mod):
    from paper_1508_03235_b300 import noc
    assert set(oracle_mod.STAT_NAMES) | {"cycle", "in_flight"} == set(noc.STATS_FIELDS)
