"""Seeded synthetic sparse matrices with band, block and scattered structure.

Shared by the tests and the benchmark; it draws random numbers and lays out
coordinates, and holds none of the products it is used to check.  RNG: numpy
PCG64 (``np.random.default_rng(seed)``).  Every generator returns a dict with
``m, n, row, col, val`` (int32 / int32 / float32 COO with unique coordinates;
where two structures hit the same cell the first-generated entry is kept) and
a ``meta`` dict describing what was planted.

The matrices stand in for the SuiteSparse matrices of the paper's evaluation
(absent here): shapes and mixes follow the ranges of its tables -- block
densities 56-100 %, block coverage 8-99 %, band coverage up to 92 %.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np


def _values(rng, size, dist):
    if dist == "normal":
        return rng.standard_normal(size, dtype=np.float32)
    if dist == "int":
        return rng.integers(-4, 5, size).astype(np.float32)
    return rng.uniform(-1.0, 1.0, size).astype(np.float32)


def _dedupe(n, parts_r: List[np.ndarray], parts_c: List[np.ndarray], parts_v: List[np.ndarray]):
    r = np.concatenate(parts_r).astype(np.int64) if parts_r else np.zeros(0, np.int64)
    c = np.concatenate(parts_c).astype(np.int64) if parts_c else np.zeros(0, np.int64)
    v = np.concatenate(parts_v).astype(np.float32) if parts_v else np.zeros(0, np.float32)
    key = r * n + c
    _, first = np.unique(key, return_index=True)   # first occurrence of each cell
    first.sort()
    return r[first].astype(np.int32), c[first].astype(np.int32), v[first]


def band_cells(m, n, offset, start, length):
    """Cells (i, i + offset) for i in [start, start + length) inside the matrix."""
    i = np.arange(start, min(m, start + length), dtype=np.int64)
    j = i + offset
    keep = (j >= 0) & (j < n)
    return i[keep], j[keep]


def block_cells(rng, r0, c0, nr, nc, density):
    if density >= 1.0:
        ii, jj = np.meshgrid(np.arange(nr), np.arange(nc), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
    else:
        mask = rng.random((nr, nc)) < density
        ii, jj = np.nonzero(mask)
    return (ii + r0).astype(np.int64), (jj + c0).astype(np.int64)


def disjoint_starts(rng, total, sides):
    """Start positions for segments of the given sides, in random order, pairwise
    disjoint inside [0, total), with random gaps."""
    k = len(sides)
    free = total - int(sum(sides))
    if free < 0:
        raise ValueError("blocks do not fit")
    order = rng.permutation(k)
    cuts = np.sort(rng.integers(0, free + 1, k))
    starts = np.empty(k, dtype=np.int64)
    pos = 0
    prev = 0
    for rank, b in enumerate(order):
        pos += int(cuts[rank]) - prev
        prev = int(cuts[rank])
        starts[b] = pos
        pos += int(sides[b])
    return starts


def powerlaw_lengths(rng, size, alpha=2.0, kmax=2000):
    """Row lengths k in [1, kmax] with P(k) proportional to k^-alpha."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    p = k ** (-alpha)
    p /= p.sum()
    return rng.choice(np.arange(1, kmax + 1), size=size, p=p)


def assemble(rng, m, n, bands=(), blocks=(), n_scatter=0, row_lengths=None, values="uniform"):
    """Build one matrix.

    bands:  (offset, start_row, length)
    blocks: (r0, c0, nrows, ncols, density)
    n_scatter: uniformly scattered entries; row_lengths: per-row counts of
    scattered entries with uniform columns (used instead of n_scatter).
    """
    R, C = [], []
    for (off, st, ln) in bands:
        i, j = band_cells(m, n, off, st, ln)
        R.append(i)
        C.append(j)
    for (r0, c0, nr, nc, dens) in blocks:
        i, j = block_cells(rng, r0, c0, nr, nc, dens)
        R.append(i)
        C.append(j)
    if row_lengths is not None:
        rl = np.asarray(row_lengths, dtype=np.int64)
        R.append(np.repeat(np.arange(m, dtype=np.int64), rl))
        C.append(rng.integers(0, n, int(rl.sum())))
    elif n_scatter:
        R.append(rng.integers(0, m, n_scatter))
        C.append(rng.integers(0, n, n_scatter))
    V = [_values(rng, a.size, values) for a in R]
    row, col, val = _dedupe(n, R, C, V)
    return dict(m=m, n=n, row=row, col=col, val=val)


# ---------------------------------------------------------------- the five workloads
def blocks_bands_scatter_4096(seed=1001, values="uniform"):
    """4096 x 4096: eight dense 64 x 64 blocks at 64-aligned positions on distinct,
    pairwise non-adjacent block rows and block columns (so that the block
    partitioner's disjointness rules can recover each of them), bands at
    offsets 0 and +-17 each over a random contiguous 30-90 % of the rows, and
    0.1 % uniformly scattered entries.  Values U[-1, 1]."""
    rng = np.random.default_rng(seed)
    n = 4096
    br = 2 * rng.choice(n // 128, 8, replace=False)
    bc = 2 * rng.choice(n // 128, 8, replace=False)
    blocks = [(int(a) * 64, int(b) * 64, 64, 64, 1.0) for a, b in zip(br, bc)]
    bands = []
    for off in (0, 17, -17):
        ln = int(rng.integers(int(0.3 * n), int(0.9 * n) + 1))
        st = int(rng.integers(0, n - ln + 1))
        bands.append((off, st, ln))
    A = assemble(rng, n, n, bands=bands, blocks=blocks, n_scatter=int(0.001 * n * n),
                 values=values)
    A["meta"] = dict(bands=bands, blocks=blocks, name="blocks+bands+scatter 4096^2")
    return A


def bands_powerlaw_1m(seed=1002, n=1_000_000, values="normal"):
    """1M x 1M: nine bands at offsets {0, +-1, +-2, +-1000, +-1001}, each over a
    random contiguous 20-100 % of the rows, plus ~5M scattered entries whose
    per-row counts follow P(k) ~ k^-2 on [1, 2000] with uniform columns.
    Values N(0, 1)."""
    rng = np.random.default_rng(seed)
    bands = []
    for off in (0, 1, -1, 2, -2, 1000, -1000, 1001, -1001):
        ln = int(rng.integers(int(0.2 * n), n + 1))
        st = int(rng.integers(0, n - ln + 1))
        bands.append((off, st, ln))
    rl = powerlaw_lengths(rng, n)
    A = assemble(rng, n, n, bands=bands, row_lengths=rl, values=values)
    A["meta"] = dict(bands=bands, name="9 bands + power-law scatter 1M^2")
    return A


def blocks_scatter_200k(seed=1003, n=200_000, block_nnz=12_000_000, n_scatter=18_000_000,
                        side=(16, 256), density=0.8, values="uniform"):
    """200k x 200k: variable-size blocks (each side uniform in 16..256, cells
    present with probability 0.8) on pairwise disjoint row and column ranges,
    holding ~40 % of the entries, plus uniformly scattered entries (~30M
    total).  Values U[-1, 1]."""
    rng = np.random.default_rng(seed)
    sides_r, sides_c = [], []
    expect = 0.0
    while expect < block_nnz:
        a, b = int(rng.integers(side[0], side[1] + 1)), int(rng.integers(side[0], side[1] + 1))
        sides_r.append(a)
        sides_c.append(b)
        expect += a * b * density
    rs = disjoint_starts(rng, n, sides_r)
    cs = disjoint_starts(rng, n, sides_c)
    blocks = [(int(r), int(c), a, b, density) for r, c, a, b in zip(rs, cs, sides_r, sides_c)]
    A = assemble(rng, n, n, blocks=blocks, n_scatter=n_scatter, values=values)
    A["meta"] = dict(blocks=blocks, name="blocks + scatter 200k^2")
    return A


def mixed_matrix(rng, m, nnz_per_row, values="uniform", side_max=256):
    """One matrix of the batched and planner workloads: its target entries per
    row are split at random (Dirichlet(1,1,1)) among bands, blocks and scatter."""
    f = rng.dirichlet([1.0, 1.0, 1.0])
    n = m
    bands = []
    nb = int(round(f[0] * nnz_per_row))
    if nb > 0:
        center = int(rng.integers(-m // 4, m // 4 + 1))
        offs = [center + k - nb // 2 for k in range(nb)]
        for off in offs:
            ln = int(rng.integers(int(0.3 * m), m + 1))
            st = int(rng.integers(0, m - ln + 1))
            bands.append((off, st, ln))
    blocks = []
    target = f[1] * nnz_per_row * m
    if target > 0 and m >= 64:
        smax = max(16, min(side_max, m // 8))
        sr, sc, got = [], [], 0.0
        while got < target and sum(sr) + smax < m and sum(sc) + smax < m:
            a, b = int(rng.integers(16, smax + 1)), int(rng.integers(16, smax + 1))
            sr.append(a)
            sc.append(b)
            got += a * b * 0.8
        if sr:
            rs, cs = disjoint_starts(rng, m, sr), disjoint_starts(rng, n, sc)
            blocks = [(int(r), int(c), a, b, 0.8) for r, c, a, b in zip(rs, cs, sr, sc)]
    ns = int(round(f[2] * nnz_per_row * m))
    A = assemble(rng, m, n, bands=bands, blocks=blocks, n_scatter=ns, values=values)
    A["meta"] = dict(bands=bands, blocks=blocks, fractions=f.tolist())
    return A


def batch_512(seed=1004, count=512, rows=(1000, 64000), npr=(5.0, 200.0), values="uniform"):
    """Many matrices of uneven size: rows log-uniform in [1k, 64k], entries per
    row log-uniform in [5, 200], mixed band / block / scatter structure."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(rows[0]), math.log(rows[1])))))
        t = float(math.exp(rng.uniform(math.log(npr[0]), math.log(npr[1]))))
        out.append(mixed_matrix(rng, m, t, values=values))
    return out


def dense_operand(seed, rows, cols=None, dist="uniform"):
    """x (cols=None) or B (rows x cols, row-major) with the stated distribution."""
    rng = np.random.default_rng(seed)
    shape = (rows,) if cols is None else (rows, cols)
    if dist == "normal":
        return rng.standard_normal(shape, dtype=np.float32)
    if dist == "int":
        return rng.integers(-4, 5, shape).astype(np.float32)
    return rng.uniform(-1.0, 1.0, shape).astype(np.float32)


def planner_matrix(rng, rows=(100_000, 1_000_000), npr=(4.0, 24.0)):
    """One matrix of the planner's data set: rows log-uniform in `rows`, entries
    per row log-uniform in `npr`, split by Dirichlet(0.7, 0.7, 0.7) shares among
    bands (up to 24 adjacent diagonals around a random offset, spans 30-100 %),
    delta-dense blocks (sides 16-512, cell density 0.6-1.0, disjoint rows and
    columns) and power-law (alpha = 2) scattered rows."""
    m = int(round(math.exp(rng.uniform(math.log(rows[0]), math.log(rows[1])))))
    npr_ = float(math.exp(rng.uniform(math.log(npr[0]), math.log(npr[1]))))
    f = rng.dirichlet([0.7, 0.7, 0.7])
    bands = []
    nb = min(24, int(round(f[0] * npr_)))
    if nb > 0:
        center = int(rng.integers(-m // 4, m // 4 + 1))
        for k in range(nb):
            ln = int(rng.integers(int(0.3 * m), m + 1))
            off = center + k - nb // 2
            ln = min(ln, m - abs(off))
            bands.append((off, int(rng.integers(0, m - abs(off) - ln + 1)), ln))
    blocks = []
    target = f[1] * npr_ * m
    smax = max(16, min(512, m // 16))
    sr, sc, got = [], [], 0.0
    dens = float(rng.uniform(0.6, 1.0))
    while got < target and sum(sr) + smax < m and sum(sc) + smax < m:
        a, b = int(rng.integers(16, smax + 1)), int(rng.integers(16, smax + 1))
        sr.append(a)
        sc.append(b)
        got += a * b * dens
    if sr:
        rs, cs = disjoint_starts(rng, m, sr), disjoint_starts(rng, m, sc)
        blocks = [(int(r), int(c), a, b, dens) for r, c, a, b in zip(rs, cs, sr, sc)]
    ns = f[2] * npr_
    rl = None
    if ns > 0.05:
        rl = powerlaw_lengths(rng, m, kmax=500)
        rl = np.minimum(500, np.round(rl * (ns / 3.4)).astype(np.int64))   # mean of P(k)~k^-2 on [1,500] ~ 3.4
    A = assemble(rng, m, m, bands=bands, blocks=blocks, row_lengths=rl, values="normal")
    A["meta"] = dict(bands=len(bands), blocks=len(blocks), fractions=f.tolist(), npr=npr_)
    return A


def planner_set_matrix(i, seed=1005, rows=(100_000, 1_000_000)):
    """Matrix i of the planner's data set (each index seeded on its own)."""
    return planner_matrix(np.random.default_rng([seed, i]), rows)
