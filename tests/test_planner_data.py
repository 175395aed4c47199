"""The learned planner's committed data set and weights, checked on the CPU.

The data set holds, for every generated matrix, its device features and the
measured SpMV / SpMM time of every candidate plan; the weights were trained on
the first matrices with the library's MLP kernels.  Here the weights are run
through the FP64 reference MLP (oracle/ml.py) on the held-out matrices: the
chosen plans must beat every fixed rule (the three-format plan, CSR alone, the
best single candidate on the training matrices) on every op, and come within
5 % of the exhaustive planner on average for SpMV and for SpMM."""
import json
import os

import numpy as np
import pytest

from oracle import ml
from paper_2407_00829_gb300 import planner as pl

HERE = os.path.dirname(pl.__file__)
DATA = os.path.join(HERE, "planner_data.npz")
WEIGHTS = os.path.join(HERE, "planner_weights.json")
N_TEST = 200


def _data():
    d = dict(np.load(DATA))
    assert list(d["names"]) == pl.NAMES and list(d["ops"]) == [o for o, _ in pl.OPS]
    return d


def test_data_set_is_consistent():
    d = _data()
    M = d["features"].shape[0]
    assert M >= N_TEST + 200
    assert d["features"].shape == (M, pl.NFEAT) and d["times"].shape == (M, len(pl.NAMES), len(pl.OPS))
    assert np.all(np.isfinite(d["features"])) and np.all(d["times"] > 0)
    idx = d["meta"][:, 0]
    assert np.all(np.diff(idx) > 0)                       # matrices in generator order, each once
    X, Y = pl.design(d)
    assert X.shape == (M * len(pl.OPS), pl.N_IN)
    assert np.all(Y >= 0) and np.allclose(Y.min(axis=1), 0)


def test_committed_weights_through_the_reference_mlp():
    d = _data()
    w = json.load(open(WEIGHTS))
    assert w["names"] == pl.NAMES and w["n_in"] == pl.N_IN
    shape = (pl.N_IN, w["hidden"], w["hidden"], len(pl.NAMES))
    X, _ = pl.design(d)
    M, O = d["features"].shape[0], len(pl.OPS)
    cut = M - N_TEST
    pred = np.mean([ml.mlp_forward(shape, np.array(p, np.float64), X[cut * O:]) for p in w["params"]], axis=0)
    picks = np.argmin(pred, axis=1).reshape(N_TEST, O)
    T = d["times"]
    q = pl.quality(T[cut:], picks)
    Yt = np.log(T[:cut] / T[:cut].min(axis=1, keepdims=True))          # [train, candidates, ops]
    best_fixed = np.argmin(np.exp(Yt).mean(axis=0), axis=0)             # per op
    fixed = {"default": np.full(O, pl.NAMES.index(pl.DEFAULT)), "csr": np.zeros(O, np.int64),
             "best_fixed": best_fixed}
    bound = {"spmv": 0.05, "spmm64_bf16": 0.05}
    for o, (op, _) in enumerate(pl.OPS):
        assert q[:, o].mean() <= bound[op], (op, q[:, o].mean())
        for name, c in fixed.items():
            qf = pl.quality(T[cut:], np.full((N_TEST, O), c[o]))
            assert q[:, o].mean() < qf[:, o].mean(), (op, name)


def test_model_selection_never_sees_the_held_out_matrices(monkeypatch):
    """planner.select scores its grid on a validation part of the training
    matrices and trains the chosen setting on the training matrices only (a
    stand-in for the device-trained ensemble records what each fit sees)."""
    d = _data()
    M, O = d["features"].shape[0], len(pl.OPS)
    fits = []

    class Fake:
        def __init__(self, seed=0, members=5, hidden=64):
            self.members = members

        def fit(self, X, Y, steps=2000, lr=2e-3):
            fits.append((X.shape[0], self.members, steps, lr, X.copy()))
            return [0.0]

        def choose(self, X):   # a rule that depends on the inputs: the candidate of the largest feature
            return np.argmax(X[:, : len(pl.NAMES)], axis=1)

    monkeypatch.setattr(pl, "LearnedPlanner", Fake)
    X, _ = pl.design(d)
    n_val = 80
    res, _ = pl.select(d, n_test=N_TEST, n_val=n_val)
    grid = pl.GRID
    assert len(fits) == len(grid) + 1
    for (rows, members, steps, lr, Xf), g in zip(fits, grid):
        assert rows == (M - N_TEST - n_val) * O
        assert (members, steps, lr) == (g["members"], g["steps"], g["lr"])
        np.testing.assert_array_equal(Xf, X[:rows])
    rows, members, steps, lr, Xf = fits[-1]
    assert rows == (M - N_TEST) * O
    np.testing.assert_array_equal(Xf, X[:rows])
    chosen = res["selection"]["chosen"]
    assert (members, steps, lr) == (chosen["members"], chosen["steps"], chosen["lr"])
    assert chosen == grid[int(np.argmin(res["selection"]["validation_loss"]))]
