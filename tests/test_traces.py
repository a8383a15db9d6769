"""Trace-file input: the text and .npz formats round-trip, addresses become
(line | write << 31) words, malformed files are rejected, and a trace drives
the oracle to issue exactly the references it lists."""
import numpy as np
import pytest

from paper_1508_03235_b300 import traces as T


def sample_traces(n_cores=4, per=50, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cores):
        lines = rng.integers(0, 5000, size=per).astype(np.uint32)
        writes = (rng.random(per) < 0.3).astype(np.uint32) << np.uint32(31)
        out.append(lines | writes)
    out[2] = out[2][:0]                      # a core with no references
    return out


def test_encoding():
    assert T.encode(0x1000, False) == 0x1000 // 64
    assert T.encode(0x1000 + 63, True) == (64 | (1 << 31))
    with pytest.raises(ValueError):
        T.encode(64 << 26, False)


@pytest.mark.parametrize("ext", [".txt", ".npz"])
def test_round_trip(tmp_path, ext):
    t = sample_traces()
    path = str(tmp_path / ("trace" + ext))
    (T.write_npz if ext == ".npz" else T.write_text)(path, t)
    back = T.load(path, len(t))
    assert len(back) == len(t)
    for a, b in zip(t, back):
        assert a.dtype == b.dtype and (a == b).all()


def test_text_errors(tmp_path):
    p = tmp_path / "bad.txt"
    for body in ("0 X 0x40\n", "9 R 0x40\n", "0 R\n", "0 R -64\n"):
        p.write_text(body)
        with pytest.raises(ValueError):
            T.read_text(str(p), 4)
    p.write_text("# only a comment\n\n1 w 128   # trailing comment\n")
    t = T.read_text(str(p), 2)
    assert len(t[0]) == 0 and list(t[1]) == [2 | (1 << 31)]


def test_trace_drives_oracle(oracle_mod):
    t = sample_traces(n_cores=4, per=40)
    p = T.trace_params(2, 2, t, period=2)
    assert p["remote_lines"] == max(int((a & ~T.WRITE_BIT).max()) for a in t if len(a)) + 1
    o = oracle_mod.OracleSim(p)
    T.apply(o, t)
    o.step(40_000)
    st = o.stats()
    assert st["refs"] == sum(len(a) for a in t)        # every listed reference, no more
    assert o.drain(100_000) >= 0
    assert o.stats()["in_flight"] == 0
