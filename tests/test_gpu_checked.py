"""The checked build (noc_set_checks): the single-writer check on the LSPD
directory.  On valid runs it changes nothing -- counters and full state hash
equal the oracle's, with directory searches, deletions and migrations
happening all the time -- and a directory message delivered to a tile that
is not its line's directory tile, which the production builds would act on,
ends the step with NOC_ERR_OWNER at that message's cycle."""
import pytest

from paper_1508_03235_b300 import inputs as I

pytestmark = pytest.mark.gpu
NOC_ERR_OWNER = 9


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def busy_params(w, h, policy, seed, **opts):
    """Tiny caches against a large address mix: L1 and L2 victims and
    directory searches and deletions every few cycles."""
    cache = I.cache_cfg(l1_ways=4, l2_ways=8, mig_window=4, mig_threshold=2, svc_q=512, **opts)
    cache.update(l1_sets=4, l2_sets=2)
    traf = I.traffic(period=2, write=0.35, priv=0.35, shared=0.35, priv_kb=2, shared_mb=0)
    traf.update(shared_lines=300, remote_lines=4_000)
    return I.sim_params(w, h, policy=policy, cache=cache, traf=traf, seed=seed)


def migrating_params(w, h, seed):
    """A hot shared region read through a 1 KB L1: the same requester keeps
    returning to the same remote block, so blocks migrate (DIRUPD at the
    directory tile)."""
    cache = I.cache_cfg(l1_kb=1, l1_ways=4, l2_kb=2, l2_ways=8, mig_window=4, mig_threshold=2, svc_q=512)
    traf = I.traffic(period=3, priv=0.3, shared=0.6, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=100, remote_lines=20_000)
    return I.sim_params(w, h, policy=2, cache=cache, traf=traf, seed=seed)


# name: (params, tiling, migrations expected)
CASES = {
    "interleaved_8x8": (dict(I.MESH_8["params"]), None, False),
    "lspd_local": (busy_params(9, 7, 1, 11), None, False),
    "lspd_migrate": (migrating_params(9, 7, 12), None, True),
    "directory_node": (busy_params(9, 7, 2, 13, dir_central=1, dir_tile=20), None, False),
    "lspd_migrate_448_threads": (busy_params(21, 21, 2, 14), (1, 1), False),
}


@pytest.mark.parametrize("name", list(CASES))
def test_checked_build_changes_nothing(noc, oracle_mod, name):
    p, tiling, migrating = CASES[name]
    g = noc.Sim(p, tiling=tiling)
    g.set_checks(True)
    o = oracle_mod.OracleSim(p)
    for n in (1300, 900):
        g.step(n)
        o.step(n)
        assert g.variant() == dict(loop="plain", kind="general", bounds=(4, 8) if p["l2_ways"] <= 8 else (4, 16))
        assert g.launch_bound() == 448
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (name, k, gs[k], v)
    assert g.state_hash() == o.state_hash(), name
    if p["policy"]:
        assert os_["dir_search"] > 200, os_
    if migrating:
        assert os_["migrations"] > 0, os_
    # the traced loop, drains and two tiles per thread are refused while checks are on
    with pytest.raises(noc.NocError):
        g.step(10, trace=True)
    g.set_checks(False)
    g.step(100)
    o.step(100)
    assert g.state_hash() == o.state_hash(), name
    o.close()


def test_directory_message_at_the_wrong_tile(noc, oracle_mod):
    """A DA for line 5 (directory tile 5 on this 8 x 8 LSPD mesh) delivered to
    tile 9.  The production build and the oracle act on it alike (whatever
    follows, the same error or none at the same cycle); the checked build
    ends the step with NOC_ERR_OWNER when tile 9 ejects it, before anything
    the production build reports."""
    p = I.sim_params(8, 8, policy=1, seed=21)
    runs = {}
    for label, checked in (("production", False), ("checked", True)):
        g = noc.Sim(p)
        g.set_checks(checked)
        g.step(200)
        g.debug_enqueue(30, 0, dict(type="DA", src=30, dst=9, line=5, e=1))
        g.step_async(400)
        runs[label] = g.error()
        g.close()
    o = oracle_mod.OracleSim(p)
    o.step(200)
    o.debug_enqueue(30, 0, dict(type="DA", src=30, dst=9, line=5, e=1))
    o.step(400, check=False)
    assert runs["production"] == o.error()
    code, cycle = runs["checked"]
    assert code == NOC_ERR_OWNER and 200 < cycle < 600, runs
    if runs["production"][0]:
        assert cycle <= runs["production"][1], runs
    o.close()
