"""The learned planner on the device.

* Training: the library's MLP kernels fit the committed timings of the
  training matrices (with the setting chosen on a validation part of them);
  on the 200 held-out matrices the chosen plans gain over every fixed rule
  (the three-format plan, which is the method without the learned part, CSR
  alone, the best single candidate) and are within 5 % of the exhaustive
  planner's on average, for SpMV and for SpMM.
* Inference: the committed weights, run by the library's forward kernel on
  the committed device features, pick the same plans as when they were saved.
* Live: on fresh matrices (not in the data set) the learned planner's plan,
  chosen from features computed on the device, is timed against every
  candidate (the exhaustive planner).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_00829_gb300 import planner as pl
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(pl.__file__)
DATA = os.path.join(HERE, "planner_data.npz")
WEIGHTS = os.path.join(HERE, "planner_weights.json")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


BOUND = {"spmv": 0.05, "spmm64_bf16": 0.05}


def _data():
    return dict(np.load(DATA))


def test_training_on_device_gains_over_fixed_plans():
    with open(WEIGHTS) as f:
        chosen = json.load(f)["eval"]["selection"]["chosen"]
    res, _ = pl.evaluate(_data(), n_test=200, seed=0, **chosen)
    for op, _ in pl.OPS:
        assert res["learned"][op]["mean_loss"] <= BOUND[op], res
        for rule in ("default", "csr", "best_fixed"):
            assert res["learned"][op]["mean_loss"] < res[rule][op]["mean_loss"], (rule, res)
            assert res["learned"]["time_ratio"][op] < res[rule]["time_ratio"][op], (rule, res)


def test_committed_weights_pick_recorded_plans():
    lp = pl.LearnedPlanner.load(WEIGHTS)
    d = _data()
    res, _ = pl.evaluate(d, n_test=200, lp=lp)
    with open(WEIGHTS) as f:
        saved = json.load(f)["eval"]
    for op, _ in pl.OPS:
        assert res["learned"][op]["mean_loss"] == pytest.approx(saved["learned"][op]["mean_loss"], abs=2e-3)
        assert res["learned"][op]["mean_loss"] <= BOUND[op]


@pytest.mark.slow
def test_live_learned_plan_close_to_exhaustive():
    lp = pl.LearnedPlanner.load(WEIGHTS)
    ratios = []
    for i in (100_000, 100_001, 100_002):
        A = synth.planner_set_matrix(i, rows=(100_000, 300_000))
        best, t, _ = pl.exhaustive(A, op=0)
        pick = pl.NAMES.index(lp.plan(A, N=0))
        ratios.append(t[pick] / t[best])
    assert np.median(ratios) <= 1.25, ratios   # three timed matrices: a loose sanity bound
