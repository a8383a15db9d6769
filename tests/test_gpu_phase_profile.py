"""The per-phase clock profile of the plain loop: turning it on runs another
build of the loop, which must give the same results (counters, histograms,
full state hash, equal to the oracle), and its sums must add up: one count per
warp and simulated cycle, every phase a positive number of clocks."""
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


@pytest.mark.parametrize("name,params,tiling,warps,kinds", [
    ("mesh8_one_cta", dict(I.MESH_8["params"]), (1, 1), 2, ("interleaved", "interleaved")),
    # an LSPD migration configuration is profiled on the base build
    ("lspd_four_ctas", I.sim_params(16, 12, policy=2, seed=9,
                                    traf=I.traffic(period=3, priv=0.4, shared=0.5, shared_mb=1)),
     (2, 2), 4 * 2, ("base", "lspd-migrate")),
])
def test_profile_changes_nothing_and_adds_up(noc, oracle_mod, name, params, tiling, warps, kinds):
    g = noc.Sim(params, tiling=tiling)
    g.set_phase_profile(True)
    o = oracle_mod.OracleSim(params)
    for n in (700, 900):
        g.step(n)
        o.step(n)
    prof = g.phase_profile()
    assert prof["warp_cycles"] == warps * 1600, prof
    for ph in noc.Sim.PHASES:
        assert prof[ph] > 0, (ph, prof)
    assert g.launch_bound() == 384
    assert g.variant()["kind"] == kinds[0]
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        assert gs[k] == v, (k, gs[k], v)
    assert g.state_hash() == o.state_hash()
    assert (g.hist(0) == o.hist(0)).all() and (g.hist(1) == o.hist(1)).all()
    # read once: cleared
    assert g.phase_profile()["warp_cycles"] == 0
    # off again: the production build, same results
    g.set_phase_profile(False)
    g.step(300)
    o.step(300)
    assert g.phase_profile()["warp_cycles"] == 0
    assert g.variant()["kind"] == kinds[1]
    assert g.state_hash() == o.state_hash()


def test_profile_refuses_ctas_beyond_its_build(noc):
    """The profiled build takes CTAs of at most 384 threads: a 21 x 21 mesh in
    one CTA (441 threads, the wide build's range) is NOC_ERR_ARG while the
    profile is on, and runs once it is off."""
    g = noc.Sim(I.sim_params(21, 21, seed=3), tiling=(1, 1), tiles_per_thread=1)
    g.set_phase_profile(True)
    with pytest.raises(noc.NocError) as e:
        g.step(10)
    assert e.value.code == 1 and "profiled loop" in str(e.value)
    g.set_phase_profile(False)
    g.step(10)
    assert g.launch_bound() == 448 and g.stats()["cycle"] == 10
