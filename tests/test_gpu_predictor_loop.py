"""The learned predictor attached to a 3-D Cahn-Hilliard plan: schedule of exact
judges and predictions, missed-block accounting, and accuracy against the dense
run.  The predictor has no counterpart in the paper; these are properties of
the scheduling rule declared in the C ABI (exact judge every J steps and at the
first step, predictions every K steps in between)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

DIMS, BLOCK, MAP = (64, 64, 64), (8, 8, 8), (8, 8, 8)
K, J, STEPS = 20, 100, 400


def _constant_predictor(bias):
    """All weights zero, head bias `bias`: p = sigmoid(bias) for every block."""
    from paper_2609_03922_gb300 import spdba
    n = int(spdba.lib().spdba_predictor_num_params())
    params = np.zeros(n, dtype=np.float32)
    params[-1] = bias
    return spdba.Predictor(MAP, max_batch=1, params=params)


def _run(mode, pred=None, seed=W.BASE_SEED + 90):
    from paper_2609_03922_gb300 import spdba
    c0 = W.ch_initial_condition(DIMS, mean=0.1, seed=seed).astype(np.float32)
    plan = spdba.Plan(DIMS, BLOCK, threshold=1e-6, reassess=10, mode=mode)
    if pred is not None:
        plan.attach_predictor(pred, K, J, 0.5)
    plan.set_field(c0)
    plan.step(STEPS)
    f = plan.get_field().astype(np.float64)
    st = plan.get_stats()
    plan.close()
    return f, st


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_schedule_and_all_active_prediction():
    """p = 1 everywhere: every predicted state is ACTIVE, so no block can be
    missed; judges run at multiples of J, predictions at the other multiples of K,
    and the result is at least as close to dense as the exact adaptive run."""
    f_dense, _ = _run(0)
    f_exact, s_exact = _run(1)
    f_pred, s_pred = _run(1, _constant_predictor(20.0))
    # every state setting counts as an assessment; the exact scans are the rest
    assert s_pred["assessments"] == STEPS // K
    assert s_pred["predictions"] == STEPS // K - STEPS // J
    assert s_pred["missed_blocks"] == 0
    assert s_pred["active_ratio_sum"] >= s_exact["active_ratio_sum"]
    assert _rel(f_pred, f_dense) <= _rel(f_exact, f_dense) + 1e-7


def test_all_frozen_prediction_is_caught_by_the_judges():
    """p = 0 everywhere: predictions freeze every block but the forced k = 0 block
    and its neighbours, so the exact judges find the blocks the prediction froze."""
    _, s_exact = _run(1)
    _, s_pred = _run(1, _constant_predictor(-20.0))
    assert s_pred["missed_blocks"] > 0
    assert s_pred["active_ratio_sum"] < s_exact["active_ratio_sum"]


def test_trained_predictor_halves_the_scans():
    """Trained on traces of two other seeds: the exact scans drop from one per
    reassessment to one per judge, few blocks are missed, and the field stays
    within the FP32 path's tolerance of the dense run."""
    import torch
    from paper_2609_03922_gb300 import predictor_train as PT
    traces = [PT.collect_trace(DIMS, BLOCK,
                               W.ch_initial_condition(DIMS, mean=0.1, seed=W.BASE_SEED + 95 + i).astype(np.float32),
                               STEPS) for i in range(2)]
    pr = PT.TrainedPredictor(MAP, max_batch=4, seed=0)
    xs, ys = [], []
    for tr in traces:
        x, y = PT.make_inputs(pr, tr, PT.build_samples(tr, K, J))
        xs.append(x)
        ys.append(y)
    hist = PT.train(pr, torch.cat(xs), torch.cat(ys), epochs=30, lr=3e-3)
    assert hist[-1] < hist[0]
    f_dense, _ = _run(0)
    f_exact, s_exact = _run(1)
    f_pred, s_pred = _run(1, pr)
    assert s_exact["assessments"] == STEPS // 10 and s_exact["predictions"] == 0
    assert s_pred["assessments"] - s_pred["predictions"] == STEPS // J
    nblocks = int(np.prod([d // b for d, b in zip(DIMS, BLOCK)]))
    assert s_pred["missed_blocks"] <= 0.05 * nblocks * (STEPS // J)
    assert _rel(f_pred, f_dense) <= 1e-4


def test_predictions_drive_the_staged_half_form():
    """128^3, Hermitian half-spectrum form with the staged update, where the
    paired z forward lists its live tiles at every state setting, predicted or
    exact.  An all-ACTIVE prediction misses no block and stays at least as close
    to the dense run as the exact adaptive run; an all-FROZEN one is caught by
    the judges."""
    from paper_2609_03922_gb300 import spdba
    dims = (128, 128, 128)
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED + 96).astype(np.float32)

    def run(mode, bias=None):
        plan = spdba.Plan(dims, BLOCK, threshold=1e-2, reassess=10, mode=mode, half_spectrum=1, fuse_update=0)
        if bias is not None:
            n = int(spdba.lib().spdba_predictor_num_params())
            params = np.zeros(n, dtype=np.float32)
            params[-1] = bias
            plan.attach_predictor(spdba.Predictor((16, 16, 16), max_batch=1, params=params), K, J, 0.5)
        plan.set_field(c0)
        plan.step(STEPS)
        f = plan.get_field().astype(np.float64)
        st = plan.get_stats()
        plan.close()
        return f, st

    f_dense, _ = run(0)
    f_exact, s_exact = run(1)
    f_all, s_all = run(1, 20.0)
    _, s_none = run(1, -20.0)
    assert s_all["predictions"] == STEPS // K - STEPS // J
    assert s_all["missed_blocks"] == 0
    assert _rel(f_all, f_dense) <= _rel(f_exact, f_dense) + 1e-7
    assert s_none["missed_blocks"] > 0
    assert s_none["active_ratio_sum"] < s_exact["active_ratio_sum"]
