"""Host-side pieces of the surrogate: feature and target definitions (S-1..S-3
readings), the relative-error floors, and the screening recall (no GPU)."""
import math

import numpy as np

from paper_1508_03235_b300 import surrogate as S


def test_screen_recall_of_perfect_inverted_and_random_pickers():
    rng = np.random.default_rng(0)
    true = rng.normal(size=(1000, 3))
    rec, rnd, best = S.screen(true.copy(), true, k=50, top_frac=0.01, random_draws=400)
    assert rec == 1.0 and len(best) == 10
    assert abs(rnd - 50 / 1000) < 0.015          # k/n in expectation
    rec, _, _ = S.screen(-true, true, k=50, top_frac=0.01)
    assert rec == 0.0
    # maximising instead of minimising picks the other end
    rec, _, best_max = S.screen(true, true, k=10, top_frac=0.01, minimise=False)
    assert rec == 1.0 and set(best_max) == set(np.argsort(-true[:, 0])[:10].tolist())


def test_targets_follow_the_metric_definitions():
    st = dict(l2lat_sum=600, l2lat_cnt=4, deflections=30, ejected=60, cycle=100)
    y = S.targets(st, tiles=64)
    assert y[0] == math.log(150.0) and y[1] == 0.5 and y[2] == 60 / (64 * 100)


def test_relative_error_floors():
    true = np.array([[math.log(100.0), 0.0, 0.0], [math.log(10.0), 2.0, 0.5]])
    pred = np.array([[math.log(110.0), 0.001, 0.0001], [math.log(10.0), 1.0, 0.25]])
    err = S.relative_errors(pred, true)
    assert np.allclose(err[0], [0.1, 0.001 / 0.01, 0.0001 / 1e-3])
    assert np.allclose(err[1], [0.0, 0.5, 0.5])
