"""The capacity model (Table 4): per-tile state bytes come from the library's
own arena layout, grow affinely with the tile count, and the tile count is
capped by the 16-bit tile indices of a flit."""
import ctypes as C

import pytest

from paper_1508_03235_b300 import capacity
from paper_1508_03235_b300 import inputs as I
from paper_1508_03235_b300 import noc


def test_arena_affine_in_tiles():
    for label, over, pol in capacity.table4_rows():
        sizes = [(64, 64), (128, 128), (255, 257)]
        b = [capacity.arena_bytes(capacity.params_for(w, h, over, pol)) for w, h in sizes]
        n = [w * h for w, h in sizes]
        slope = (b[2] - b[0]) / (n[2] - n[0])
        mid = b[0] + slope * (n[1] - n[0])
        assert abs(mid - b[1]) < 256 * 32, label        # 256-byte alignment of each array


def test_rows_are_table4_and_fit_b300():
    rows = capacity.table4_rows()
    assert [(o["l1_sets"], o["l1_ways"], o["l2_sets"], o["l2_ways"]) for _, o, _ in rows] == [
        (128, 4, 512, 8), (128, 4, 128, 4), (32, 2, 32, 2), (32, 2, 32, 2)]
    assert [p for _, _, p in rows] == [I.POLICY_LSPD_MIGRATE] * 3 + [I.POLICY_LSPD_LOCAL]
    per = []
    for _, over, pol in rows:
        per_tile, by_mem, n = capacity.capacity(over, pol, 270e9)
        per.append(per_tile)
        assert n == capacity.MAX_TILES and by_mem > capacity.MAX_TILES
    # smaller caches and no migration history need less state per tile
    assert per[0] > per[1] > per[2] > per[3]


def test_tile_count_cap():
    p = I.sim_params(256, 256)
    h = C.c_void_p()
    rc = noc.lib().noc_create(256, 256, C.byref(noc.cache_struct(p)), 0,
                              C.byref(noc.traffic_struct(p)), 1, C.byref(h))
    assert noc.ERR_NAMES[rc] == "NOC_ERR_ARG"
    w, hh = capacity.LARGEST_MESH
    assert w * hh == capacity.MAX_TILES
