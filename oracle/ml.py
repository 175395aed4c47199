"""FP64 references for the learned planner's device code.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``features`` -- the structural features the library's feature kernels
  compute (definitions in the library's sable_ml.cu header comment), from the
  COO arrays with plain numpy counting; exact when nnz <= 2^22 (no sampling).
* ``mlp_forward`` / ``mlp_grad`` -- the MLP n_in -> h1 (ReLU) -> h2 (ReLU) ->
  n_out (linear) with masked mean squared error, parameters in the library's
  flat layout, gradient by the chain rule written out layer by layer.
* ``adam`` -- one bias-corrected Adam step (Kingma & Ba).
"""
from __future__ import annotations

import numpy as np

NFEAT = 24


def features(m: int, n: int, row, col) -> np.ndarray:
    row = np.asarray(row, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    nnz = row.size
    out = np.zeros(NFEAT)
    rl = np.bincount(row, minlength=m).astype(np.float64) if m else np.zeros(0)
    mean = rl.mean() if m else 0.0
    var = max(0.0, (rl * rl).mean() - mean * mean) if m else 0.0
    out[0] = np.log2(m + 1.0) / 24
    out[1] = np.log2(n + 1.0) / 24
    out[2] = np.log2(nnz + 1.0) / 32
    out[3] = np.log2(mean + 1.0) / 8
    out[4] = (np.sqrt(var) / mean if mean > 0 else 0.0) / 8
    out[5] = np.log2((rl.max() if m else 0) + 1.0) / 16
    if m:
        L = rl.astype(np.int64)
        bins = np.where(L == 0, 0, np.minimum(7, 1 + np.floor(np.log2(np.maximum(L, 1))).astype(np.int64)))
        out[6:14] = np.bincount(bins, minlength=8)[:8] / m
    if nnz:
        d = col - row
        cnt = np.bincount(d + m - 1, minlength=m + n - 1)
        per_entry = cnt[d + m - 1]
        mn = max(1, min(m, n))
        b = np.where(per_entry * 64 < mn, 0, np.where(per_entry * 16 < mn, 1, np.where(per_entry * 4 < mn, 2, 3)))
        out[14:18] = np.bincount(b, minlength=4) / nnz
        out[18] = np.count_nonzero(np.abs(d) <= 64) / nnz
        stride = max(1, -(-nnz // (1 << 22)))
        s = np.arange(0, nnz, stride)
        key = (row[s] >> 3) * ((n + 7) // 8) + (col[s] >> 3)
        uk, inv, kc = np.unique(key, return_inverse=True, return_counts=True)
        c = kc[inv]
        out[19:23] = [np.mean(c >= 48), np.mean(c >= 32), np.mean(c >= 16), np.mean(c >= 8)]
    out[23] = 0.0
    return out


def _split(shape, p):
    n_in, h1, h2, n_out = shape
    o = 0
    W1 = p[o:o + n_in * h1].reshape(n_in, h1); o += n_in * h1
    b1 = p[o:o + h1]; o += h1
    W2 = p[o:o + h1 * h2].reshape(h1, h2); o += h1 * h2
    b2 = p[o:o + h2]; o += h2
    W3 = p[o:o + h2 * n_out].reshape(h2, n_out); o += h2 * n_out
    b3 = p[o:o + n_out]; o += n_out
    return W1, b1, W2, b2, W3, b3


def mlp_forward(shape, params, X):
    W1, b1, W2, b2, W3, b3 = _split(shape, np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1 + b1
    A1 = np.maximum(Z1, 0)
    Z2 = A1 @ W2 + b2
    A2 = np.maximum(Z2, 0)
    return A2 @ W3 + b3


def mlp_loss(shape, params, X, T, mask=None):
    Y = mlp_forward(shape, params, X)
    M = np.ones_like(Y) if mask is None else np.asarray(mask, dtype=np.float64)
    return float(np.sum(M * (Y - np.asarray(T, dtype=np.float64)) ** 2) / max(M.sum(), 1.0))


def mlp_grad(shape, params, X, T, mask=None):
    """(loss, gradient in the flat parameter layout)."""
    p = np.asarray(params, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = _split(shape, p)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1 + b1
    A1 = np.maximum(Z1, 0)
    Z2 = A1 @ W2 + b2
    A2 = np.maximum(Z2, 0)
    Y = A2 @ W3 + b3
    M = np.ones_like(Y) if mask is None else np.asarray(mask, dtype=np.float64)
    D = max(M.sum(), 1.0)
    R = Y - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(M * R * R) / D)
    dY = 2.0 * M * R / D
    dW3 = A2.T @ dY
    db3 = dY.sum(0)
    dA2 = dY @ W3.T
    dZ2 = dA2 * (Z2 > 0)
    dW2 = A1.T @ dZ2
    db2 = dZ2.sum(0)
    dA1 = dZ2 @ W2.T
    dZ1 = dA1 * (Z1 > 0)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def adam(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
