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


def test_features_sizes_and_row_length_bins_by_hand():
    # 36 rows of 200 columns; row-length bin k (0, 1, 2-3, 4-7, 8-15, 16-31,
    # 32-63, >= 64) gets k + 1 rows, with both ends of every bin used, so each
    # share is distinct and a shifted bin edge moves a row between bins
    lengths = [0, 1, 1, 2, 3, 3, 4, 5, 6, 7, 8, 9, 15, 15, 12, 16, 17, 31, 31, 20, 25,
               32, 33, 63, 63, 40, 50, 60, 64, 65, 100, 128, 199, 70, 80, 90]
    m, n = len(lengths), 200
    row = np.repeat(np.arange(m), lengths)
    col = np.concatenate([np.arange(L) for L in lengths])
    nnz = int(sum(lengths))
    f = ml.features(m, n, row, col)
    assert f[0] == pytest.approx(np.log2(37.0) / 24, rel=1e-15)      # m = 36
    assert f[1] == pytest.approx(np.log2(201.0) / 24, rel=1e-15)     # n = 200
    assert f[2] == pytest.approx(np.log2(nnz + 1.0) / 32, rel=1e-15)
    assert nnz == 1368
    np.testing.assert_allclose(f[6:14], np.arange(1, 9) / 36.0, rtol=0, atol=1e-15)
    mean = 1368 / 36
    sd = np.sqrt(sum(L * L for L in lengths) / 36 - mean * mean)
    assert f[3] == pytest.approx(np.log2(mean + 1) / 8, rel=1e-14)
    assert f[4] == pytest.approx(sd / mean / 8, rel=1e-12)
    assert f[5] == pytest.approx(np.log2(200.0) / 16, rel=1e-15)     # longest row 199


def test_features_diagonal_count_bins_by_hand():
    # 256 x 256: min(m, n) = 256, so M[d] < 4 is bin 14, < 16 bin 15, < 64
    # bin 16, >= 64 bin 17.  Diagonals with counts on both sides of each
    # threshold: 3 | 4, 15 | 16, 63 | 64 (and 200)
    m = n = 256
    counts = {5: 3, -7: 4, 9: 15, 11: 16, -20: 63, 30: 64, 0: 200}
    row, col = [], []
    for d, c in counts.items():
        i0 = max(0, -d)
        for i in range(i0, i0 + c):
            row.append(i)
            col.append(i + d)
    nnz = sum(counts.values())
    f = ml.features(m, n, np.array(row), np.array(col))
    assert f[14] == pytest.approx(3 / nnz, rel=1e-15)
    assert f[15] == pytest.approx((4 + 15) / nnz, rel=1e-15)
    assert f[16] == pytest.approx((16 + 63) / nnz, rel=1e-15)
    assert f[17] == pytest.approx((64 + 200) / nnz, rel=1e-15)
    assert f[18] == 1.0                                   # every |d| <= 64


def test_features_near_diagonal_edge_and_tile_thresholds():
    # |j - i| <= 64 counts, 65 does not
    m = n = 300
    row = np.array([0, 0, 10, 100, 200])
    col = np.array([64, 65, 10, 35, 136])                 # d = 64, 65, 0, -65, -64
    f = ml.features(m, n, row, col)
    assert f[18] == pytest.approx(3 / 5, rel=1e-15)
    # 8 x 8 tiles holding 47 | 48, 31 | 32, 15 | 16, 7 | 8 entries: each
    # entry takes its tile's count, so the share of entries in tiles with
    # >= 48 is 48 / total, >= 32 is (48 + 47 + 32) / total, and so on
    tile_counts = [47, 48, 31, 32, 15, 16, 7, 8]
    row, col = [], []
    for t, c in enumerate(tile_counts):
        cells = [(8 * t + a // 8, 8 * t + a % 8) for a in range(c)]
        row += [r for r, _ in cells]
        col += [q for _, q in cells]
    tot = sum(tile_counts)
    f = ml.features(64, 64, np.array(row), np.array(col))
    assert f[19] == pytest.approx(48 / tot, rel=1e-15)
    assert f[20] == pytest.approx((47 + 48 + 32) / tot, rel=1e-15)
    assert f[21] == pytest.approx((47 + 48 + 31 + 32 + 16) / tot, rel=1e-15)
    assert f[22] == pytest.approx((tot - 7) / tot, rel=1e-15)
