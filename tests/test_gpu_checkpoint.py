"""Checkpoint and resume: a run saved at some cycle and restored (into the
same handle, or a fresh one of the same configuration) continues exactly as
the uninterrupted run does -- per-cycle hashes, counters, histograms, full
state hash -- and equals the oracle."""
import numpy as np
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


def lspd_params():
    cache = I.cache_cfg(l1_kb=2, l1_ways=2, l2_kb=8, l2_ways=4, mig_window=4, mig_threshold=2, svc_q=512)
    traf = I.traffic(period=3, priv=0.35, shared=0.5, priv_kb=4, shared_mb=0)
    traf.update(shared_lines=400, remote_lines=20_000)
    return I.sim_params(12, 10, policy=2, cache=cache, traf=traf, seed=21)


def end_state(s):
    return s.stats(), s.state_hash(), s.hist(0).tolist(), s.hist(1).tolist()


@pytest.mark.parametrize("name", ["mesh8", "lspd_migrate", "two_tiles"])
def test_resume_equals_uninterrupted_run(noc, oracle_mod, name):
    p = dict(I.MESH_8["params"]) if name == "mesh8" else lspd_params()
    kw = dict(tiling=(2, 2), tiles_per_thread=2 if name == "two_tiles" else None)
    a = noc.Sim(p, **kw)
    a.step(1500)
    image = a.save()
    a.step(1200)
    want = end_state(a)
    # the same handle, restored
    a.load(image)
    assert a.stats()["cycle"] == 1500
    a.step(1200)
    assert end_state(a) == want
    # a fresh handle of the same configuration
    b = noc.Sim(p, **kw)
    b.load(image)
    b.step(700)
    b.step(500)
    assert end_state(b) == want
    o = oracle_mod.OracleSim(p)
    o.step(2700)
    assert all(want[0][k] == v for k, v in o.stats().items())
    assert want[1] == o.state_hash()


def test_resume_per_cycle_hashes_and_drain(noc, oracle_mod):
    p = lspd_params()
    a = noc.Sim(p, tiling=(3, 2))
    a.step(900)
    image = a.save()
    b = noc.Sim(p, tiling=(2, 3))                # another tiling: results never depend on it
    b.load(image)
    o = oracle_mod.OracleSim(p)
    o.step(900)
    tg, to = b.step(400, trace=True), o.step(400, trace=True)
    assert (tg == to).all()
    assert b.drain(100_000) == o.drain(100_000)
    assert b.state_hash() == o.state_hash()
    # a drain's reference stop is part of the image
    img2 = b.save()
    c = noc.Sim(p)
    c.load(img2)
    c.step(50)
    assert c.stats()["refs"] == b.stats()["refs"]


def test_foreign_images_are_refused(noc):
    a = noc.Sim(I.MESH_8["params"])
    a.step(10)
    image = a.save()
    other = noc.Sim(dict(I.MESH_8["params"], seed=2))
    with pytest.raises(noc.NocError):
        other.load(image)
    with pytest.raises(noc.NocError):
        a.load(np.zeros(64, dtype=np.uint8))
