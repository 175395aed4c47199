"""Pins for the FP64 oracle: each check ties the oracle to something other than
itself (dense FP64 matmul, exact integer arithmetic, the paper's worked
examples, brute force on tiny inputs, closed forms)."""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import extract as ox
from oracle import formats as of
import synth
from conftest import read_golden


def _dense(m, n, row, col, val):
    A = np.zeros((m, n), dtype=np.float64)
    np.add.at(A, (row, col), val.astype(np.float64))
    return A


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spmv_spmm_match_dense_matmul(seed):
    rng = np.random.default_rng(seed)
    m, n, nnz = 37, 29, 300                      # duplicates occur at this density
    row = rng.integers(0, m, nnz).astype(np.int32)
    col = rng.integers(0, n, nnz).astype(np.int32)
    val = rng.uniform(-1, 1, nnz).astype(np.float32)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    B = rng.uniform(-1, 1, (n, 7)).astype(np.float32)
    A = _dense(m, n, row, col, val)
    ref_y = torch.from_numpy(A) @ torch.from_numpy(x.astype(np.float64))
    ref_C = torch.from_numpy(A) @ torch.from_numpy(B.astype(np.float64))
    np.testing.assert_allclose(oracle.spmv(m, row, col, val, x), ref_y.numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(oracle.spmm(m, row, col, val, B), ref_C.numpy(), rtol=1e-12, atol=1e-13)
    sel = np.array([0, 5, 36, 5])
    np.testing.assert_allclose(oracle.spmm_rows(m, row, col, val, B, sel), ref_C.numpy()[sel],
                               rtol=1e-12, atol=1e-13)


def test_integer_inputs_are_exact():
    rng = np.random.default_rng(7)
    m, n, nnz = 50, 40, 400
    row = rng.integers(0, m, nnz)
    col = rng.integers(0, n, nnz)
    val = rng.integers(-4, 5, nnz)
    x = rng.integers(-4, 5, n)
    B = rng.integers(-4, 5, (n, 5))
    want_y = [0] * m
    want_C = [[0] * 5 for _ in range(m)]
    for i, j, a in zip(row.tolist(), col.tolist(), val.tolist()):
        want_y[i] += a * int(x[j])
        for c in range(5):
            want_C[i][c] += a * int(B[j, c])
    y = oracle.spmv(m, row, col, val.astype(np.float32), x.astype(np.float32))
    C = oracle.spmm(m, row, col, val.astype(np.float32), B.astype(np.float32))
    assert y.tolist() == [float(v) for v in want_y]
    assert C.tolist() == [[float(v) for v in r] for r in want_C]


def test_special_cases():
    n = 64
    d = np.arange(1, n + 1, dtype=np.float32)
    x = np.linspace(-1, 1, n).astype(np.float32)
    i = np.arange(n)
    np.testing.assert_array_equal(oracle.spmv(n, i, i, d, x), d.astype(np.float64) * x)
    y0 = oracle.spmv(10, np.zeros(0, int), np.zeros(0, int), np.zeros(0, np.float32),
                     np.ones(5, np.float32))
    assert y0.tolist() == [0.0] * 10
    # one dense block reduces to a GEMV
    rng = np.random.default_rng(3)
    blk = rng.uniform(-1, 1, (12, 9)).astype(np.float32)
    ii, jj = np.meshgrid(np.arange(12) + 20, np.arange(9) + 5, indexing="ij")
    xx = rng.uniform(-1, 1, 30).astype(np.float32)
    y = oracle.spmv(40, ii.ravel(), jj.ravel(), blk.ravel(), xx)
    ref = (torch.from_numpy(blk.astype(np.float64)) @ torch.from_numpy(xx[5:14].astype(np.float64))).numpy()
    np.testing.assert_allclose(y[20:32], ref, rtol=1e-13)
    assert not np.any(y[:20]) and not np.any(y[32:])


def test_normwise_err():
    assert oracle.normwise_err([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert oracle.normwise_err([1.0, 2.5], [1.0, 2.0]) == pytest.approx(0.25)
    assert oracle.normwise_err([0.0], [0.0]) == 0.0


def test_bf16_round_matches_torch_and_ties():
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(100000).astype(np.float32) * 1000,
                        rng.uniform(-1e-30, 1e-30, 1000).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, 3.0e38, -3.0e38], np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(a).view(np.uint32), ref.view(np.uint32))
    # halfway cases: 1 + 2^-8 lies between 1 and 1 + 2^-7 -> ties to even (1.0);
    # 1 + 3*2^-8 lies between 1+2^-7 and 1+2^-6 -> ties to even (1 + 2^-6)
    t = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8], np.float32)
    assert oracle.bf16_round(t).tolist() == [1.0, 1 + 2.0 ** -6]


def test_pow2_scale():
    assert oracle.pow2_scale(1.0) == 1.0
    assert oracle.pow2_scale(0.75) == 1.0
    assert oracle.pow2_scale(1.5) == 2.0
    assert oracle.pow2_scale(4.0) == 4.0
    assert oracle.pow2_scale(0.0) == 1.0
    for v in [1e-20, 3.7, 1234.5, 2.0 ** -130]:
        s = oracle.pow2_scale(v)
        assert s >= v > s / 2 and math.log2(s) == int(math.log2(s))


# ------------------------------------------------------------------ formats
def _entries_from_dense(M):
    return {(i, j): v for i, r in enumerate(M) for j, v in enumerate(r) if v != 0}


def test_vdia_layout_fig4():
    g = read_golden("vdia_fig4.txt")
    ent = _entries_from_dense(g["matrix"])
    segs = [(1, 4, [-1, 0, 1]), (6, 3, [-6, -5, -4, -3])]
    arr = of.vdia_arrays(ent, 10, segs)
    for k in ("val", "idiag", "seg_row_start", "seg_nrows", "seg_ndiags", "seg_val_ptr",
              "seg_idiag_ptr"):
        assert [float(v) for v in arr[k]] == g[k], k


def test_vbr_layout_fig7():
    g = read_golden("vbr_fig9.txt")
    M = g["matrix"]
    ent = {(i, j): v for i, r in enumerate(M) for j, v in enumerate(r)}   # zeros inside blocks kept
    bp, bindx = [int(v) for v in g["Bpntrb"]], [int(v) for v in g["Bindx"]]
    stored = [(bi, bindx[k]) for bi in range(len(bp) - 1) for k in range(bp[bi], bp[bi + 1])]
    arr = of.vbr_arrays(ent, [int(v) for v in g["Rpntr"]], [int(v) for v in g["Cpntr"]], stored)
    for k in ("Val", "Indx", "Bindx", "Rpntr", "Cpntr", "Bpntrb"):
        assert [float(v) for v in arr[k]] == g[k], k
    # every nonzero of the matrix lies in a stored block: SpMV through VBR = dense
    x = np.arange(1, 12, dtype=np.float64)
    y = np.zeros(11)
    R, Cp, Val, Indx = arr["Rpntr"], arr["Cpntr"], arr["Val"], arr["Indx"]
    for bi in range(5):
        for k in range(bp[bi], bp[bi + 1]):
            bj = arr["Bindx"][k]
            nr = R[bi + 1] - R[bi]
            for c in range(Cp[bj], Cp[bj + 1]):
                for r in range(R[bi], R[bi + 1]):
                    y[r] += Val[Indx[k] + (c - Cp[bj]) * nr + (r - R[bi])] * x[c]
    np.testing.assert_array_equal(y, np.array(M) @ x)


# ------------------------------------------------------------------ extractors
def _coo_from_dense(M):
    M = np.asarray(M)
    r, c = np.nonzero(M)
    return r, c, M[r, c].astype(np.float32)


def test_band_extractor_recovers_fig4():
    g = read_golden("vdia_fig4.txt")
    r, c, v = _coo_from_dense(g["matrix"])
    p = ox.Params(delta=0.75, a_min=12, l_seg=3, count_min=3)
    ex = ox.run_plan(10, 10, r, c, v, [(ox.VDIA, p), (ox.CSR, None)])
    assert ex.segments == [(1, 4, -1, 3), (6, 3, -6, 4)]
    assert np.all(ex.owner == ox.VDIA)
    ent = _entries_from_dense(g["matrix"])
    arr = of.vdia_arrays(ent, 10, [(r0, nr, list(range(lo, lo + nd))) for r0, nr, lo, nd in ex.segments])
    assert [float(x) for x in arr["val"]] == g["val"]
    assert [float(x) for x in arr["idiag"]] == g["idiag"]


def test_fit_ribbon_cases():
    # row 5 of a 1 x 20 style matrix: entries at columns 3,4,5,6 and 9
    ent = [(5, 3), (5, 4), (5, 5), (5, 6), (5, 9)]
    R = ox.Residual(10, 20, np.array([e[0] for e in ent]), np.array([e[1] for e in ent]),
                    np.arange(len(ent)))
    assert ox.fit_ribbon(R, 5, 0, 0.75, 64) == (2, 1, 4)        # 3..6 full; 9 would give 5/7
    assert ox.fit_ribbon(R, 5, 0, 0.7, 64) == (2, 4, 5)         # 5/7 >= 0.7 reaches column 9
    assert ox.fit_ribbon(R, 5, 1, 0.75, 64) == (3, 0, 4)        # centre 6, grows below
    assert ox.fit_ribbon(R, 5, 2, 0.75, 64) == (0, 0, 0)        # no entry at column 7
    assert ox.fit_ribbon(R, 5, 0, 0.75, 1) == (1, 1, 3)         # w_max caps both sides


def test_planted_band_is_one_segment():
    rng = np.random.default_rng(5)
    A = synth.assemble(rng, 300, 300, bands=[(o, 40, 200) for o in (-2, -1, 0, 1, 2)])
    ex = ox.run_plan(300, 300, A["row"], A["col"], A["val"],
                     [(ox.VDIA, ox.Params(delta=0.75, a_min=100)), (ox.CSR, None)])
    assert ex.segments == [(40, 200, -2, 5)]
    assert np.all(ex.owner == ox.VDIA)


@pytest.mark.parametrize("tile", [0, 8])
def test_planted_full_block_is_recovered(tile):
    rng = np.random.default_rng(9)
    A = synth.assemble(rng, 90, 80, blocks=[(21, 13, 30, 25, 1.0)])
    p = ox.Params(delta=0.5, a_min=300, tile=tile, max_span=64)
    ex = ox.run_plan(90, 80, A["row"], A["col"], A["val"], [(ox.VBR, p), (ox.CSR, None)])
    assert ex.blocks == [(21, 30, 13, 25)]
    assert np.all(ex.owner == ox.VBR)


def test_coverage_cutoff_rejects_small_share():
    rng = np.random.default_rng(9)
    A = synth.assemble(rng, 200, 200, blocks=[(21, 13, 20, 20, 1.0)], n_scatter=6000)
    p = ox.Params(delta=0.5, a_min=300, tile=8, max_span=64)   # 400 of ~6300 < 8 %
    ex = ox.run_plan(200, 200, A["row"], A["col"], A["val"], [(ox.VBR, p), (ox.CSR, None)])
    assert ex.blocks == [] and np.all(ex.owner == ox.CSR)


def _brute_best(Mb, a_min, delta, s_min):
    m, n = Mb.shape
    best = -1.0
    P = np.zeros((m + 1, n + 1), dtype=np.int64)
    P[1:, 1:] = np.cumsum(np.cumsum(Mb, 0), 1)
    for r0 in range(m):
        for r1 in range(r0 + s_min, m + 1):
            for c0 in range(n):
                for c1 in range(c0 + 1, n + 1):
                    a = (r1 - r0) * (c1 - c0)
                    if a < a_min:
                        continue
                    z = P[r1, c1] - P[r0, c1] - P[r1, c0] + P[r0, c0]
                    d = z / a
                    if d >= delta:
                        best = max(best, a * math.pow(d - delta, 1.5))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_find_block_bounded_by_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 12, 12
    Mb = (rng.random((m, n)) < rng.uniform(0.3, 0.8)).astype(np.int64)
    r, c = np.nonzero(Mb)
    R = ox.Residual(m, n, r, c, np.arange(r.size))
    p = ox.Params(delta=0.5, a_min=12, max_span=12)
    sc2, o0, o1, i0, i1 = ox.find_block(R.rowlist, 0, m, 0, n, p)   # sc2: the score squared
    best = _brute_best(Mb, p.a_min, p.delta, ox._isqrt_ceil(p.a_min))
    assert sc2 <= best * best * (1 + 1e-12) + 1e-12
    # every one of these matrices holds a delta-dense window (brute force finds
    # one), and Algorithm 2 must return some window then
    assert best > 0 and sc2 > 0
    a = (o1 - o0) * (i1 - i0)
    z = int(Mb[o0:o1, i0:i1].sum())
    assert math.isclose(math.sqrt(sc2), a * math.pow(z / a - p.delta, 1.5), rel_tol=1e-12, abs_tol=1e-12)
    assert a >= p.a_min and z / a >= p.delta and o1 - o0 >= ox._isqrt_ceil(p.a_min)


def _lines(Mb):
    r, c = np.nonzero(Mb)
    return ox.Residual(Mb.shape[0], Mb.shape[1], r, c, np.arange(r.size))


@pytest.mark.parametrize("m,n,span", [(20, 15, 64), (30, 8, 64), (40, 12, 25)])
def test_find_block_all_ones_closed_form(m, n, span):
    # Algorithm 2 on a region with every cell set: every window has density 1,
    # so the score a (1 - delta)^1.5 grows with the area and the best window is
    # the widest and tallest one the outer span cap allows, from the first start
    R = _lines(np.ones((m, n), dtype=np.int64))
    p = ox.Params(delta=0.5, a_min=36, max_span=span)
    sc2, o0, o1, i0, i1 = ox.find_block(R.rowlist, 0, m, 0, n, p)
    h = min(m, span)
    a = h * n
    assert (o0, o1, i0, i1) == (0, h, 0, n)
    assert sc2 == pytest.approx((a * (1 - p.delta)) ** 3 / a, rel=1e-15)


@pytest.mark.parametrize("r0,h,w,n", [(0, 12, 10, 30), (7, 10, 12, 25), (3, 20, 9, 9), (11, 16, 16, 40)])
def test_find_block_planted_block_at_inner_start(r0, h, w, n):
    # a full h x w block whose columns start at the region's first inner index:
    # the window scan cannot carry empty columns in front of it, so Algorithm 2
    # returns exactly the block, whose score is the brute-force maximum over
    # every rectangle (adding empty cells lowers a (d - delta)^1.5 for d >= delta)
    m = 40
    Mb = np.zeros((m, n), dtype=np.int64)
    Mb[r0:r0 + h, 0:w] = 1
    p = ox.Params(delta=0.5, a_min=90, max_span=64)
    sc2, o0, o1, i0, i1 = ox.find_block(_lines(Mb).rowlist, 0, m, 0, n, p)
    assert (o0, o1, i0, i1) == (r0, r0 + h, 0, w)
    brute = _brute_best(Mb, p.a_min, p.delta, ox._isqrt_ceil(p.a_min))
    assert sc2 > 0 and math.isclose(math.sqrt(sc2), brute, rel_tol=1e-12)
    assert math.isclose(math.sqrt(sc2), h * w * (1 - p.delta) ** 1.5, rel_tol=1e-12)


@pytest.mark.parametrize("r0,c0,h,w", [(5, 7, 12, 10), (20, 30, 15, 20), (3, 25, 20, 5), (30, 3, 10, 37)])
def test_find_block_window_covers_planted_block_and_trim_recovers_it(r0, c0, h, w):
    # elsewhere the literal window may keep empty columns or rows around the
    # block (the sliding window of Algorithm 2 stops at the first dense
    # window), but it always covers the block with a positive score, and Trim
    # (Algorithm 1) strips exactly the empty lines back off
    m, n = 60, 50
    Mb = np.zeros((m, n), dtype=np.int64)
    Mb[r0:r0 + h, c0:c0 + w] = 1
    R = _lines(Mb)
    p = ox.Params(delta=0.5, a_min=100, max_span=64)
    for lines, O, I, (br0, br1, bc0, bc1) in ((R.rowlist, m, n, (r0, r0 + h, c0, c0 + w)),
                                              (R.collist, n, m, (c0, c0 + w, r0, r0 + h))):
        if br1 - br0 < ox._isqrt_ceil(p.a_min):
            continue                     # block shorter than s_min along this search's outer axis
        sc2, o0, o1, i0, i1 = ox.find_block(lines, 0, O, 0, I, p)
        assert sc2 > 0
        assert o0 <= br0 and br1 <= o1 and i0 <= bc0 and bc1 <= i1
        win = (o0, o1, i0, i1) if lines is R.rowlist else (i0, i1, o0, o1)
        assert ox.trim(R, *win) == (r0, r0 + h, c0, c0 + w, h * w)


def test_candidate_regions_band_slabs_by_hand():
    # A band of the 9 diagonals -4..4 over 200 rows, 8 x 8 cells, delta 0.5:
    # a diagonal cell holds 5+6+7+8+8+7+6+5 = 52 >= 32 entries (hot), an
    # off-diagonal cell 1+2+3+4 = 10 (cold), so the hot cells are (I, I) for
    # I = 0..24, one 8-connected component of 25 cells in a 25 x 25 box
    # (4 x 25 < 625: under a quarter full) and taller than S = 64 / 8 = 8 cell
    # rows.  It is cut into slabs of 8 cell rows from its first row: cell rows
    # [0,8), [8,16), [16,24), [24,25); each box is its cells' columns grown by
    # one cell on each side, and grown outward in rows only at the first and
    # last slab (clipped to the matrix); no two boxes overlap, so none merge.
    m = 200
    r, c = [], []
    for i in range(m):
        for d in range(-4, 5):
            if 0 <= i + d < m:
                r.append(i)
                c.append(i + d)
    R = ox.Residual(m, m, np.array(r), np.array(c), np.arange(len(r)))
    p = ox.Params(delta=0.5, a_min=100, max_span=64, tile=8)
    cells = [(0, 8, 0, 9), (8, 16, 7, 17), (16, 24, 15, 25), (24, 25, 23, 25)]
    expect = [(8 * a, min(m, 8 * b), 8 * cc, min(m, 8 * d)) for (a, b, cc, d) in cells]
    assert ox.candidate_regions(R, p) == expect


def test_candidate_regions_band_inside_matrix_by_hand():
    # the diagonals -4..4 over rows 40..159 of a 240 x 240 matrix: hot cells
    # (I, I) for I = 5..19 (15 cells, box 15 x 15 = 225 > 4 x 15), taller
    # than S = 8 cell rows, so two slabs: cell rows [5, 13) and [13, 20).  The
    # first slab grows up by one cell row (to 4), the last down by one (to
    # 21); columns are each slab's cells grown by one: [4, 14) and [12, 21).
    m = 240
    r, c = [], []
    for i in range(40, 160):
        for d in range(-4, 5):
            r.append(i)
            c.append(i + d)
    R = ox.Residual(m, m, np.array(r), np.array(c), np.arange(len(r)))
    p = ox.Params(delta=0.5, a_min=100, max_span=64, tile=8)
    assert ox.candidate_regions(R, p) == [(32, 104, 32, 112), (104, 168, 96, 168)]


def test_candidate_regions_tall_component_over_a_quarter_full_is_one_box():
    # an L of full cells: columns 0..7 over all 200 rows (cells (I, 0), I =
    # 0..24) and rows 192..199 over columns 0..23 (cells (24, 0..2)): 27 cells
    # in a 25 x 3 box, 27 / 75 = 36 % >= a quarter, so no slab cut although it
    # is taller than S: one box, grown by one cell and clipped: rows [0, 200),
    # columns [0, 32)
    m = n = 200
    Mb = np.zeros((m, n), dtype=np.int64)
    Mb[:, 0:8] = 1
    Mb[192:200, 0:24] = 1
    p = ox.Params(delta=0.5, a_min=100, max_span=64, tile=8)
    assert ox.candidate_regions(_lines(Mb), p) == [(0, 200, 0, 32)]


def test_candidate_regions_single_block_box_by_hand():
    # one full 19 x 30 block, rows 17..35 and columns 41..70, of a 100 x 120
    # matrix, 8 x 8 cells, delta 0.5 (hot: >= 32 of 64 entries).  Cell rows
    # 2, 3, 4 hold 7, 8, 4 of its rows; cell columns 5, 6, 7, 8 hold 7, 8, 8, 7
    # of its columns.  Hot: every cell of rows 2 and 3, and in row 4 the cells
    # of columns 6 and 7 (4 x 8 = 32, exactly delta x area) but not 5 and 8
    # (4 x 7 = 28).  One component, cell rows [2, 5) x columns [5, 9), grown
    # by one cell: rows [8, 48), columns [32, 80).
    m, n = 100, 120
    Mb = np.zeros((m, n), dtype=np.int64)
    Mb[17:36, 41:71] = 1
    p = ox.Params(delta=0.5, a_min=100, max_span=64, tile=8)
    assert ox.candidate_regions(_lines(Mb), p) == [(8, 48, 32, 80)]


@pytest.mark.parametrize("tile", [0, 8])
def test_short_wide_block_found_by_the_column_search(tile):
    # 4 rows x 60 columns, a_min 100 (s_min = 10): a row-outer window needs 10
    # rows, so its density is at most 4 / 10 < delta and the CSR search finds
    # nothing; the CSC search (columns outer, 60 >= 10) finds the block, and
    # Decompose must take it (Algorithm 1 keeps the better of the two)
    m, n = 50, 90
    Mb = np.zeros((m, n), dtype=np.int64)
    Mb[20:24, 15:75] = 1
    r, c = np.nonzero(Mb)
    p = ox.Params(delta=0.5, a_min=100, max_span=64, tile=tile)
    ex = ox.run_plan(m, n, r, c, np.ones(r.size, dtype=np.float32), [(ox.VBR, p), (ox.CSR, None)])
    assert ex.blocks == [(20, 4, 15, 60)]


@pytest.mark.parametrize("seed", range(3))
def test_prepass_equals_algorithm1_per_box_and_recovers_planted_blocks(seed):
    # The candidate-region pre-pass is not in the paper.  What it must do:
    # (1) recover full planted blocks that lie far apart (the ground truth
    # here, independent of any implementation), and (2) give exactly what
    # literal Algorithm 1 (tile = 0) gives when run on each candidate box's
    # submatrix alone.  (Literal Algorithm 1 on the whole matrix can lose a
    # block to the "row or column already used" rule, so it is not the
    # reference for the whole matrix.)
    rng = np.random.default_rng(400 + seed)
    m = n = 160
    planted = [(4, 6, 20, 24), (60, 70, 30, 18), (120, 120, 25, 30)]
    A = synth.assemble(rng, m, n, blocks=[(r0, c0, nr, nc, 1.0) for (r0, c0, nr, nc) in planted], n_scatter=150)
    p8 = ox.Params(delta=0.5, a_min=300, max_span=64, tile=8)
    ex = ox.run_plan(m, n, A["row"], A["col"], A["val"], [(ox.VBR, p8), (ox.CSR, None)])
    assert ex.blocks == sorted((r0, nr, c0, nc) for (r0, c0, nr, nc) in planted)
    rows, cols, _ = ox.canonicalize(m, n, A["row"], A["col"], A["val"])
    R = ox.Residual(m, n, rows, cols, np.arange(rows.size))
    per_box = []
    p0 = ox.Params(delta=0.5, a_min=300, max_span=64, tile=0, coverage_min=0.0)
    for (r0, r1, c0, c1) in ox.candidate_regions(R, p8):
        sel = (rows >= r0) & (rows < r1) & (cols >= c0) & (cols < c1)
        Rb = ox.Residual(r1 - r0, c1 - c0, rows[sel] - r0, cols[sel] - c0, np.arange(int(sel.sum())))
        per_box += [(a + r0, b + r0, c + c0, d + c0) for (a, b, c, d, _) in ox.partition_blocks(Rb, p0)]
    assert sorted((a, b - a, c, d - c) for (a, b, c, d) in per_box) == ex.blocks


@pytest.mark.parametrize("threads", [False, True])
def test_row_order_spmv_is_identical_to_the_coo_loop(threads):
    # the row-loop form adds each row's terms in the COO input order, so its
    # FP64 result is bit-identical to the COO loop, with or without threads
    rng = np.random.default_rng(21)
    m, n, nnz = 5000, 3000, 60000
    row = rng.integers(0, m, nnz).astype(np.int32)
    col = rng.integers(0, n, nnz).astype(np.int32)
    val = rng.standard_normal(nnz).astype(np.float32)
    x = rng.standard_normal(n).astype(np.float32)
    ref = oracle.spmv(m, row, col, val, x)
    ro = oracle.RowOrder(m, row, col, val)
    if threads and oracle.omp_threads() == 0:
        pytest.skip("no OpenMP in this host compiler")
    y = ro.spmv(x, threads=threads)
    assert np.array_equal(y.view(np.uint64), ref.view(np.uint64))
    assert np.all(np.diff(ro.rp) >= 0) and ro.rp[-1] == nnz
    assert np.all(np.diff(row[ro.perm].astype(np.int64)) >= 0)      # grouped by row


def test_merge_segments_by_hand():
    # rows 0..9 carry offsets -1..1 (one pass), rows 5..14 offsets 40, 41
    # (another): three row ranges, [0,5) {-1,0,1}, [5,10) {-1,0,1,40,41},
    # [10,15) {40,41}; a third segment continuing the last set merges into it
    segs = [(0, 10, -1, 3), (5, 10, 40, 2), (15, 5, 40, 2)]
    assert ox.merge_segments(segs) == [(0, 5, (-1, 0, 1)), (5, 5, (-1, 0, 1, 40, 41)), (10, 10, (40, 41))]
    assert ox.merge_segments([(3, 4, 2, 1)]) == [(3, 4, (2,))]
    assert ox.merge_segments([]) == []


def test_second_band_pass_claims_far_band_on_masked_rows():
    # a main band {-1, 0, 1} and a far band {+50} on the same 200 rows.  One
    # pass of Algorithm 3: the first candidate (offset -1, ties by offset)
    # grows to the ribbon [-1, 1] on every row (the far band is 49 zero cells
    # away: density 4/52 < delta) and masks all rows, so offset 50 finds no
    # unmasked row and goes to CSR.  A second pass over that residual finds
    # the far band alone: one segment, offset 50.  The merged layout is one
    # segment with idiag [-1, 0, 1, 50] (Section 4.2.1), arrays by hand.
    m, n = 200, 260
    A = synth.assemble(np.random.default_rng(4), m, n, bands=[(-1, 0, m), (0, 0, m), (1, 0, m), (50, 0, m)],
                       values="int")
    one = ox.run_plan(m, n, A["row"], A["col"], A["val"],
                      [(ox.VDIA, ox.Params(delta=0.75, a_min=100, l_seg=16)), (ox.CSR, None)])
    assert one.segments == [(0, 200, -1, 3)]
    far = (one.cols - one.rows) == 50
    assert np.all(one.owner[far] == ox.CSR) and np.all(one.owner[~far] == ox.VDIA)
    two = ox.run_plan(m, n, A["row"], A["col"], A["val"],
                      [(ox.VDIA, ox.Params(delta=0.75, a_min=100, l_seg=16, passes=2)), (ox.CSR, None)])
    assert sorted(two.segments) == [(0, 200, -1, 3), (0, 200, 50, 1)]
    assert np.all(two.owner == ox.VDIA)
    merged = ox.merge_segments(two.segments)
    assert merged == [(0, 200, (-1, 0, 1, 50))]
    entries = {(int(i), int(j)): float(v) for i, j, v in zip(two.rows, two.cols, two.vals)}
    arr = of.vdia_arrays(entries, n, merged)
    assert arr["idiag"] == [-1, 0, 1, 50] and arr["seg_ndiags"] == [4] and arr["seg_nrows"] == [200]
    assert arr["seg_val_ptr"] == [0] and arr["seg_idiag_ptr"] == [0]
    val = arr["val"]
    assert len(val) == 800 and val[0] == 0.0                      # row 0 has no column -1
    for k, off in enumerate((-1, 0, 1, 50)):
        for r in range(m):
            c = r + off
            assert val[200 * k + r] == (entries.get((r, c), 0.0) if 0 <= c < n else 0.0)
