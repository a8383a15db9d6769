"""The largest square mesh that runs as one co-resident launch (found by a
search over sides; one thread per tile bounds it) in each of the four cache
configurations of Table 4 equals the oracle bit for bit (counters, histogram,
full state hash), and the next side up is refused with NOC_ERR_ARG."""
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


@pytest.mark.parametrize("row", range(4))
def test_largest_mesh_matches_oracle(noc, oracle_mod, row):
    label, over, pol = capacity.table4_rows()[row]
    side = capacity.largest_square(over, pol)
    assert side >= 208 and not capacity.launches(side + 1, over, pol)
    w = h = side
    p = capacity.params_for(w, h, over, pol)
    g = noc.Sim(p)
    g.step(CYCLES)
    gs, gh, g0 = g.stats(), g.state_hash(), g.hist(0)
    g.close()
    o = oracle_mod.OracleSim(p)
    o.step(CYCLES)
    os_ = o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (label, k, gs[k], v)
    assert (g0 == o.hist(0)).all(), label
    assert gh == o.state_hash(), label
    assert gs["injected"] > 0 and gs["cycle"] == CYCLES
