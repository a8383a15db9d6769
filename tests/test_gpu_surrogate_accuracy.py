"""The learned surrogate against the exact simulator, at the workload's
definitions: trained by the library's own tensor-core kernels on 2,000 design
points of the batch workload (each simulated for 20,000 cycles by the batch
engine), scored on 500 held-out points (mean relative error per output, with
the epsilon floors of the error definition), for three training seeds.

Screening: the 500 held-out points form a candidate pool whose exact outputs
are known.  The network picks the 25 candidates (5 %) it predicts to have the
lowest mean L2 access latency, the ones an exact simulation would then
confirm; the test measures what fraction of the pool's true best 1 % (5
points) those picks contain, against 25 random picks at the same simulation
budget (5 % in expectation)."""
import pytest

pytestmark = pytest.mark.gpu

MRE_MAX = 0.05


@pytest.fixture(scope="module")
def result():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import surrogate as S
    return S.evaluate(train=2_000, holdout=500, cycles=20_000, seeds=(0, 1, 2))


def test_held_out_error_within_five_percent(result):
    for run in result["runs"]:
        for name, v in run["mre"].items():
            assert v <= MRE_MAX, (run["seed"], name, v)


def test_screening_finds_the_best_designs(result):
    recalls = [r["screen_recall"] for r in result["runs"]]
    rnd = sum(r["random_recall"] for r in result["runs"]) / len(result["runs"])
    assert 0.02 < rnd < 0.08                    # k / n = 5 % for random picks
    assert min(recalls) >= 0.6 and sum(recalls) / len(recalls) >= 10 * rnd, (recalls, rnd)
