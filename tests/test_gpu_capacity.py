"""Table 4 on a B300.  For each of the four cache configurations:

* the largest square mesh that runs with one tile per thread (the fast loop;
  with CTAs of up to 448 threads that is 255 x 255, the next side up passing
  the 16-bit tile indices) equals the oracle bit for bit, and the next side up
  is refused in that loop;
* the largest mesh the 16-bit tile indices allow, 255 x 257 = 65,535 tiles,
  runs (automatically with one tile per thread: 4 x 37 rectangles of 448
  tiles, one CTA per SM) and equals the oracle bit for bit -- counters,
  flit-latency histogram and full state hash -- and so does the same run
  with two tiles per thread."""
import pytest

from paper_1508_03235_b300 import capacity

pytestmark = pytest.mark.gpu
CYCLES = 300


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def compare(noc, oracle_mod, p, label, modes=(None,)):
    """Run p for each tiles-per-thread setting in modes and compare each run
    with one oracle run; return the tiles per thread each run used."""
    o = oracle_mod.OracleSim(p)
    o.step(CYCLES)
    os_, oh, o0 = o.stats(), o.state_hash(), o.hist(0)
    o.close()
    used = []
    for m in modes:
        g = noc.Sim(p, tiles_per_thread=m)
        g.step(CYCLES)
        gs, gh, g0 = g.stats(), g.state_hash(), g.hist(0)
        used.append(g.tiles_per_thread())
        g.close()
        for k, v in os_.items():
            if k in gs:
                assert gs[k] == v, (label, m, k, gs[k], v)
        assert (g0 == o0).all(), (label, m)
        assert gh == oh, (label, m)
        assert gs["injected"] > 0 and gs["cycle"] == CYCLES
    return used


@pytest.mark.parametrize("row", range(4))
def test_largest_one_tile_mesh_matches_oracle(noc, oracle_mod, row):
    label, over, pol = capacity.table4_rows()[row]
    side = capacity.largest_square(over, pol, tiles_per_thread=1)
    assert side >= 208 and not capacity.launches(side + 1, over, pol, tiles_per_thread=1)
    assert compare(noc, oracle_mod, capacity.params_for(side, side, over, pol), label, (1,)) == [1]


@pytest.mark.parametrize("row", range(4))
def test_largest_mesh_matches_oracle(noc, oracle_mod, row):
    label, over, pol = capacity.table4_rows()[row]
    w, h = capacity.LARGEST_MESH
    assert compare(noc, oracle_mod, capacity.params_for(w, h, over, pol), label, (None, 2)) == [1, 2]
