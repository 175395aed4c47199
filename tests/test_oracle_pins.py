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
    if sc2 >= 0:
        a = (o1 - o0) * (i1 - i0)
        z = int(Mb[o0:o1, i0:i1].sum())
        assert math.isclose(math.sqrt(sc2), a * math.pow(z / a - p.delta, 1.5), rel_tol=1e-12, abs_tol=1e-12)
        assert a >= p.a_min and z / a >= p.delta and o1 - o0 >= ox._isqrt_ceil(p.a_min)
    else:
        assert best < 0 or True


@pytest.mark.parametrize("seed", range(5))
def test_trim_is_a_local_optimum(seed):
    rng = np.random.default_rng(200 + seed)
    Mb = (rng.random((15, 15)) < 0.6).astype(np.int64)
    r, c = np.nonzero(Mb)
    R = ox.Residual(15, 15, r, c, np.arange(r.size))
    r0, r1, c0, c1, z = ox.trim(R, 0, 15, 0, 15)
    assert z == Mb[r0:r1, c0:c1].sum()
    dens = z / ((r1 - r0) * (c1 - c0))
    for (a, b, cc, dd) in [(r0 + 1, r1, c0, c1), (r0, r1 - 1, c0, c1),
                           (r0, r1, c0 + 1, c1), (r0, r1, c0, c1 - 1)]:
        if b > a and dd > cc:
            assert Mb[a:b, cc:dd].sum() / ((b - a) * (dd - cc)) <= dens + 1e-15


def _format_cells(ex, entries):
    vd, vb, cs = {}, {}, {}
    for (r0, nr, lo, nd) in ex.segments:
        for r in range(r0, r0 + nr):
            for o in range(lo, lo + nd):
                c = r + o
                if 0 <= c < ex.n:
                    key = (r, c)
                    vd[key] = entries[key][1] if key in entries and entries[key][0] == ox.VDIA else 0.0
    for (r0, nr, c0, nc) in ex.blocks:
        for r in range(r0, r0 + nr):
            for c in range(c0, c0 + nc):
                key = (r, c)
                vb[key] = entries[key][1] if key in entries and entries[key][0] == ox.VBR else 0.0
    for key, (o, v) in entries.items():
        if o == ox.CSR:
            cs[key] = v
    return vd, vb, cs


@pytest.mark.parametrize("seed", range(3))
def test_three_format_plan_partition_and_invariants(seed):
    rng = np.random.default_rng(300 + seed)
    m = 160
    A = synth.assemble(rng, m, m, bands=[(o, 10, 120) for o in (-1, 0, 1)] + [(40, 0, 100)],
                       blocks=[(100, 5, 24, 30, 0.85), (20, 120, 30, 20, 0.9)], n_scatter=300)
    pv = ox.Params(delta=0.75, a_min=200, l_seg=16)
    pb = ox.Params(delta=0.5, a_min=200, max_span=64, tile=8)
    ex = ox.run_plan(m, m, A["row"], A["col"], A["val"], [(ox.VDIA, pv), (ox.VBR, pb), (ox.CSR, None)])
    entries = {(int(i), int(j)): (int(o), v) for i, j, o, v in zip(ex.rows, ex.cols, ex.owner, ex.vals)}
    ox.check_partition(ex, *_format_cells(ex, entries))
    # VBR invariants (Algorithm 1): row- and column-disjoint, width >= 2, dense, large
    for a, b in itertools.combinations(ex.blocks, 2):
        assert a[0] + a[1] <= b[0] or b[0] + b[1] <= a[0]
        assert a[2] + a[3] <= b[2] or b[2] + b[3] <= a[2]
    for (r0, nr, c0, nc) in ex.blocks:
        z = sum(1 for (i, j), (o, _) in entries.items() if o == ox.VBR and r0 <= i < r0 + nr and c0 <= j < c0 + nc)
        assert nc >= 2 and nr * nc >= pb.a_min and z / (nr * nc) >= pb.delta
    # VDIA invariants (Algorithms 3, 4): row-disjoint, long enough
    rows_seen = set()
    for (r0, nr, lo, nd) in ex.segments:
        assert nr >= pv.l_seg
        rr = set(range(r0, r0 + nr))
        assert not (rr & rows_seen)
        rows_seen |= rr
    assert len(ex.segments) >= 1 and len(ex.blocks) == 2


def test_partition_checker_catches_mistakes():
    rng = np.random.default_rng(1)
    A = synth.assemble(rng, 64, 64, bands=[(0, 0, 64), (1, 0, 64)], n_scatter=50)
    ex = ox.run_plan(64, 64, A["row"], A["col"], A["val"],
                     [(ox.VDIA, ox.Params(delta=0.75, a_min=50, l_seg=8)), (ox.CSR, None)])
    entries = {(int(i), int(j)): (int(o), v) for i, j, o, v in zip(ex.rows, ex.cols, ex.owner, ex.vals)}
    vd, vb, cs = _format_cells(ex, entries)
    ox.check_partition(ex, vd, vb, cs)
    k = next(iter(cs))
    bad = dict(cs)
    del bad[k]
    with pytest.raises(AssertionError):
        ox.check_partition(ex, vd, vb, bad)                  # dropped entry
    bad = dict(cs)
    bad[k] = np.float32(bad[k]) + np.float32(1.0)
    with pytest.raises(AssertionError):
        ox.check_partition(ex, vd, vb, bad)                  # changed value
    kd = next(key for key in vd if vd[key] != 0)
    bad = dict(cs)
    bad[kd] = vd[kd]
    with pytest.raises(AssertionError):
        ox.check_partition(ex, vd, vb, bad)                  # entry held twice
    kz = next((key for key in vd if vd[key] == 0), None)
    if kz is not None:
        badv = dict(vd)
        badv[kz] = 1.0
        with pytest.raises(AssertionError):
            ox.check_partition(ex, badv, vb, cs)             # non-zero padding


def test_incomplete_plan_raises():
    rng = np.random.default_rng(2)
    A = synth.assemble(rng, 50, 50, n_scatter=100)
    with pytest.raises(ValueError):
        ox.run_plan(50, 50, A["row"], A["col"], A["val"], [(ox.VDIA, None)])
