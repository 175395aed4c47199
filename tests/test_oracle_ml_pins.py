"""Pins for the FP64 references of the learned planner (features, MLP, Adam):
finite differences, closed forms and hand-built matrices."""
import numpy as np
import pytest

from oracle import ml

SHAPE = (6, 5, 4, 3)


def _params(seed):
    rng = np.random.default_rng(seed)
    n_in, h1, h2, n_out = SHAPE
    count = n_in * h1 + h1 + h1 * h2 + h2 + h2 * n_out + n_out
    return rng.standard_normal(count)


@pytest.mark.parametrize("seed", range(3))
def test_mlp_grad_matches_finite_differences(seed):
    rng = np.random.default_rng(10 + seed)
    p = _params(seed)
    X = rng.standard_normal((7, SHAPE[0]))
    T = rng.standard_normal((7, SHAPE[3]))
    mask = (rng.random((7, SHAPE[3])) < 0.7).astype(float)
    loss, g = ml.mlp_grad(SHAPE, p, X, T, mask)
    assert loss == pytest.approx(ml.mlp_loss(SHAPE, p, X, T, mask), rel=1e-12)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (ml.mlp_loss(SHAPE, p + e, X, T, mask) - ml.mlp_loss(SHAPE, p - e, X, T, mask)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8)


def test_mlp_bias_gradient_closed_form():
    # d loss / d b3 = 2 sum_b mask (Y - T) / sum mask, whatever the hidden layers are
    rng = np.random.default_rng(3)
    p = _params(4)
    X = rng.standard_normal((5, SHAPE[0]))
    T = rng.standard_normal((5, SHAPE[3]))
    _, g = ml.mlp_grad(SHAPE, p, X, T)
    Y = ml.mlp_forward(SHAPE, p, X)
    np.testing.assert_allclose(g[-SHAPE[3]:], 2 * (Y - T).sum(0) / Y.size, rtol=1e-12)


def test_adam_first_step_closed_form():
    # step 1: m_hat = g, v_hat = g^2, so the update is -lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = ml.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_features_hand_built():
    n = 64
    i = np.arange(n)
    f = ml.features(n, n, i, i)                     # identity
    assert f[7] == 1.0 and f[6] == 0.0              # every row has exactly one entry
    assert f[17] == 1.0 and f[18] == 1.0            # one full diagonal (count n >= n/4), all near
    assert f[3] == pytest.approx(np.log2(2.0) / 8) and f[4] == 0.0
    r, c = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    f = ml.features(32, 32, r.ravel(), c.ravel())    # one dense 16 x 16 block
    assert f[19:23].tolist() == [1.0, 1.0, 1.0, 1.0]  # every entry in a full 8 x 8 tile
    assert f[6] == 0.5                               # rows 16..31 are empty
    assert f[5] == pytest.approx(np.log2(17.0) / 16)
