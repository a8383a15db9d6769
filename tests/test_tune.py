"""Host-side logic of the autotuner and of the batch engine's kernel-variant
groups (no GPU: noc_batch_create is host-only)."""
import pytest

from paper_1508_03235_b300 import inputs as I


def test_batch_groups_follow_the_variant_rules():
    """Cache-mode instances with a class's exact ways and no option form the
    class's group of their L2 policy (interleaved 0-2, LSPD local placement
    5-7, LSPD migration 8-10); other instances without options the base
    group; any option -- the directory node among them, which the
    interleaved L2 ignores -- the general group."""
    from paper_1508_03235_b300 import noc
    base = dict(I.MESH_8["params"])
    w16 = dict(l2_ways=16, l2_sets=256)
    w1616 = dict(l1_ways=16, l1_sets=32, l2_ways=16)
    pts = [dict(base), dict(base, **w16), dict(base, **w1616),
           dict(base, policy=1), dict(base, policy=2), dict(base, l1_ways=3),
           dict(base, packet_mode=1), dict(base, policy=1, age_mode=1), dict(base, l1_write_back=1),
           dict(base, mode=I.MODE_NETWORK),
           dict(base, policy=1, **w16), dict(base, policy=1, **w1616), dict(base, policy=2, **w16),
           dict(base, policy=2, **w1616), dict(base, policy=1, dir_central=1), dict(base, dir_central=1),
           dict(base, policy=2, l2_ways=12), dict(base, policy=2, mode=I.MODE_NETWORK)]
    assert noc.batch_groups(pts) == [0, 1, 2, 5, 8, 3, 4, 4, 4, 3, 6, 7, 9, 10, 4, 0, 3, 3]


def test_design_point_groups():
    from paper_1508_03235_b300 import noc
    pts = I.batch_design_points(64, seed=0)
    for p in pts:
        p.pop("design")
    g = noc.batch_groups(pts)
    assert all(x == {0: 0, 1: 5, 2: 8}[p["policy"]] for x, p in zip(g, pts))


def test_stratified_sample_spans_the_sizes():
    from paper_1508_03235_b300 import tune
    pts = I.batch_design_points(100, seed=1)
    idx = list(range(100))
    s = tune.stratified_sample(pts, idx, 10)
    assert len(s) == len(set(s)) == 10
    sizes = sorted(pts[i]["mesh_w"] for i in idx)
    got = sorted(pts[i]["mesh_w"] for i in s)
    assert got[0] == sizes[0] and got[-1] >= sizes[90]
    assert tune.stratified_sample(pts, idx[:5], 10) == sorted(idx[:5], key=lambda i: (pts[i]["mesh_w"] ** 2, i))


def test_batch_candidates():
    from paper_1508_03235_b300 import tune
    c = tune.batch_candidates()
    assert len(c) == len(tune.BATCH_SIDES) * 2 * 3 == len(set(c))
    assert all(1 <= side and side * side <= 384 for side, _, _ in c)


def test_spread_candidates_keep_the_rectangle_shape():
    from paper_1508_03235_b300 import tune as T
    assert T.spread_candidates(208, 208, 2, 70, 148) == [(2, 71), (2, 72), (2, 73), (2, 74)]
    assert T.spread_candidates(208, 208, 2, 74, 148) == [(2, 70), (2, 71), (2, 72), (2, 73)]
    assert T.spread_candidates(8, 8, 1, 1, 148) == []
    for (W, H, gx, gy, cap) in ((208, 208, 2, 70, 148), (64, 64, 1, 32, 148), (100, 60, 4, 6, 40),
                                (255, 257, 3, 40, 148), (208, 208, 2, 73, 148)):
        out = T.spread_candidates(W, H, gx, gy, cap)
        shape = (-(-W // gx), -(-H // gy))
        assert (gx, gy) not in out and len(set(out)) == len(out)
        assert [a * b for a, b in out] == sorted(a * b for a, b in out)
        # exactly every other grid of that largest shape within the cap
        every = {(a, b) for a in range(1, W + 1) for b in range(1, H + 1)
                 if (-(-W // a), -(-H // b)) == shape and a * b <= cap}
        assert set(out) == every - {(gx, gy)}
