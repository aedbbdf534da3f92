"""The model-guided tuner (random sample, neural-network cost model, best predicted
configurations confirmed) against the exhaustive one on the same problem."""
import pytest
import torch

from paper_1605_06399_gb300 import ImclError, _abi, ops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    ops.tune_clear()
    assert ops.device_status() == 0


@pytest.mark.parametrize("k", [5, 11])
def test_model_guided_finds_a_near_best_variant(k):
    prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", k, k, 2048, 2048)
    ex = ops.tune(prob, budget_s=60.0, reps=5)
    res = ops.tune_model(prob, n_sample=24, n_confirm=8, reps=5, seed=7)
    rep = res["report"]
    assert rep["candidates"] > 24
    assert rep["sampled"] == 24 and rep["confirmed"] == 8
    assert 3 <= rep["valid"] <= 40
    assert rep["model_rmse"] >= 0.0 and rep["seconds"] > 0.0
    assert rep["holdout"] == 8 and 0 <= rep["holdout_valid"] <= 8 and rep["holdout_rmse"] >= 0.0
    timed = rep["sampled"] + rep["confirmed"] + rep["holdout"]
    assert timed < 0.3 * rep["candidates"], rep   # the wider space: a few hundred configurations
    # timing noise allowed; a model that ranked at random would often miss by far more
    assert res["best_ms"] <= 1.25 * ex["best_ms"], (res, ex)
    assert res["best_ms"] < res["plain_ms"]
    assert ops.default_variant(prob) == res["variant"]   # cached like imagecl_tune


def test_model_guided_with_nothing_to_time_returns_plain():
    prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", 3, 3, 256, 256)
    res = ops.tune_model(prob, n_sample=0, n_confirm=0, reps=2, seed=1)
    assert res["variant"]["kind"] == _abi.KIND_PLAIN
    assert res["report"]["sampled"] == 0 and res["report"]["confirmed"] == 0
    assert res["best_ms"] == res["plain_ms"]


def test_model_guided_rejects_negative_counts():
    prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", 3, 3, 64, 64)
    with pytest.raises(ImclError) as ei:
        ops.tune_model(prob, n_sample=-1)
    assert ei.value.status == _abi.ERR_INVALID
