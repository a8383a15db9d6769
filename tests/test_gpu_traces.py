"""Trace-driven runs: per-core traces read from a file drive the CUDA path
and the oracle to the same state, cycle for cycle (8x8, every cycle's hash)
and at a larger mesh (32x32, full state after a run)."""
import numpy as np
import pytest

from paper_1508_03235_b300 import traces as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def noc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import noc as _noc
    return _noc


def locality_traces(n_cores, per, seed):
    """Each core: 70% of references to its own 256-line window, 20% to 4096
    shared lines, 10% anywhere in 2^20 lines; 30% writes."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cores):
        u = rng.random(per)
        own = 8192 + c * 256 + rng.integers(0, 256, per)
        shared = rng.integers(0, 4096, per)
        far = rng.integers(0, 1 << 20, per)
        lines = np.where(u < 0.7, own, np.where(u < 0.9, shared, far)).astype(np.uint32)
        out.append(lines | ((rng.random(per) < 0.3).astype(np.uint32) << np.uint32(31)))
    return out


def same(g, o):
    gs, os_ = g.stats(), o.stats()
    for k, v in os_.items():
        if k in gs:
            assert gs[k] == v, (k, gs[k], v)
    assert g.state_hash() == o.state_hash()


@pytest.mark.parametrize("policy", [0, 2])
def test_trace_file_mesh8_every_cycle(noc, oracle_mod, tmp_path, policy):
    t = locality_traces(64, 300, seed=5 + policy)
    path = str(tmp_path / "mesh8.txt")
    T.write_text(path, t)
    t = T.load(path, 64)
    p = T.trace_params(8, 8, t, period=3, policy=policy)
    g, o = noc.Sim(p, tiling=(2, 2)), oracle_mod.OracleSim(p)
    T.apply(g, t)
    T.apply(o, t)
    tg, to = g.step(1500, trace=True), o.step(1500, trace=True)
    assert (tg == to).all()
    g.step(3000)
    o.step(3000)
    same(g, o)


def test_trace_file_mesh32(noc, oracle_mod, tmp_path):
    t = locality_traces(1024, 200, seed=11)
    path = str(tmp_path / "mesh32.npz")
    T.write_npz(path, t)
    t = T.load(path, 1024)
    p = T.trace_params(32, 32, t, period=2)
    g, o = noc.Sim(p), oracle_mod.OracleSim(p)
    T.apply(g, t)
    T.apply(o, t)
    g.step(2500)
    o.step(2500)
    same(g, o)
    assert g.stats()["refs"] > 0
