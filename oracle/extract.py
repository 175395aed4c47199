"""Reference extractors: CSR, band (VDIA) and block (VBR) partitioning.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python loops in
the order of the paper's algorithms, meant for small matrices.

Readings of the paper fixed here (the CUDA library's host code follows the
same readings, written independently):

* Canonical matrix: COO triples with duplicates summed (FP64, input order,
  then rounded once to FP32).  Explicit zeros are structural entries, since
  extraction depends only on structure (Section 3.4).
* CSRExtractor (Appendix A.1) claims every remaining entry.
* ExtractBands (Appendix D, Algorithm 3):  M[d] = residual entries on
  diagonal d = j - i (|d| <= d_max); candidates are offsets with
  M[d] >= count_min, by decreasing M[d], ties by increasing d.  A candidate
  is accepted when its segments' summed area is >= A_min and their density
  (summed entries / summed area) is >= delta; accepted rows are masked.
* FitRibbon (named in Section 4.2 and Algorithm 3, never defined).  Reading:
  if row i has no residual entry at column i + d the extent is (0, 0, 0).
  Otherwise the ribbon starts as that single cell and grows greedily: the
  two candidate growths are "reach the nearest entry below the ribbon" and
  "reach the nearest entry above it", each adding one entry and the zeros in
  between; the narrower resulting ribbon wins (below on a tie), and is taken
  only when its density stays >= delta and the side's extent stays <= w_max.
  k_i is the number of entries in the final ribbon [d - l_i, d + u_i].
* Multi-ribbon VDIA (passes > 1): Algorithm 3 runs `passes` times, each
  pass over the residual the previous one left and with its own row mask
  (Algorithm 3's used[] starts false), so a row may carry ribbons of several
  passes at different offsets, e.g. a main band and a far band whose rows a
  first pass masked.  ``merge_segments`` gives the VDIA layout of such a
  partition (Section 4.2.1: each segment carries its own list of diagonal
  offsets): the row ranges are cut at every segment boundary and each piece
  covered by the same segments becomes one segment whose offsets are the
  sorted union of theirs.
* GrowSegments (Algorithm 4), literally; "nnz at row j" counts row j's
  entries inside the current ribbon [d - L, d + U].  Segment area is
  (L + U + 1) x rows, cells outside [0, ncols) included (stored as zeros).
* Partition / Decompose / FindBlock (Section 4.1, Algorithms 1 and 2),
  literally, with (a) the density test and the score base taken as delta
  (identical to the printed 0.5 at the default delta = 0.5), (b) FindBlock's
  outer span capped at max_span, (c) ties kept by the first found in scan
  order (strict '>'; the CSR search wins a tie against the CSC search),
  (d) Trim removes, per round, the one edge (top, bottom, left, right) whose
  removal gives the largest strict density gain, first edge on a tie, until
  no removal helps, (e) width = number of columns.
* Candidate regions (a pre-pass that is not in the paper, needed to run
  Algorithm 1 on matrices with 10^5+ rows): when ``tile`` > 0 the matrix is
  cut into tile x tile cells; a cell is hot when its entries >= delta * its
  area; 8-connected hot cells form components whose bounding boxes, grown
  by one cell on each side and clipped, are merged until disjoint, sorted by
  (row, column), and Decompose runs on each box instead of on the whole
  matrix.  ``tile`` = 0 runs Algorithm 1 on the whole matrix.  A component
  spanning more than S = ceil(max_span / tile) cell rows whose cells fill
  under a quarter of its bounding box (a diagonal band) gives instead one box
  per slab of S cell rows counted from its first row: its cells' bounding box
  in that slab, grown by one cell in columns and, at the component's first and
  last slab, outward in rows.  Without the cut, a long band makes one box as
  large as the matrix and Algorithm 1's recursion along it costs
  O(rows^2 x entries per row).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

VDIA, VBR, CSR = 0, 1, 2


@dataclass
class Params:
    delta: float = 0.5
    a_min: int = 2500
    l_seg: int = 32
    d_max: int = 0          # 0: every offset
    count_min: int = 0      # 0: ceil(delta * l_seg)
    w_max: int = 64
    coverage_min: float = 0.08
    max_span: int = 512
    tile: int = 8
    passes: int = 1         # VDIA: runs of Algorithm 3 over the shrinking residual


def default_params(kind: int) -> Params:
    if kind == VDIA:
        return Params(delta=0.75)
    return Params(delta=0.5)


# ---------------------------------------------------------------- canonical form
def canonicalize(m: int, n: int, row, col, val):
    """Sorted unique (i, j) with duplicate values summed (FP64, then FP32)."""
    row = np.asarray(row, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float32)
    if row.size and (row.min() < 0 or row.max() >= m or col.min() < 0 or col.max() >= n):
        raise ValueError("COO index out of range")
    key = row * n + col
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    uniq, first = np.unique(key_s, return_index=True)
    sums = np.zeros(uniq.size, dtype=np.float64)
    grp = np.repeat(np.arange(uniq.size), np.diff(np.append(first, key_s.size)))
    v = val[order].astype(np.float64)
    for g, x in zip(grp.tolist(), v.tolist()):    # input order inside each group
        sums[g] += x
    return (uniq // n).astype(np.int64), (uniq % n).astype(np.int64), sums.astype(np.float32)


class Residual:
    """Unclaimed entries of the canonical matrix, as per-row and per-column lists."""

    def __init__(self, m: int, n: int, rows, cols, ids):
        self.m, self.n = m, n
        self.rowlist: List[List[int]] = [[] for _ in range(m)]
        self.rowids: List[List[int]] = [[] for _ in range(m)]
        self.collist: List[List[int]] = [[] for _ in range(n)]
        for i, j, e in zip(rows.tolist(), cols.tolist(), ids.tolist()):
            self.rowlist[i].append(j)
            self.rowids[i].append(e)
            self.collist[j].append(i)
        for i in range(m):
            if len(self.rowlist[i]) > 1:
                o = np.argsort(self.rowlist[i], kind="stable")
                self.rowlist[i] = [self.rowlist[i][k] for k in o]
                self.rowids[i] = [self.rowids[i][k] for k in o]
        for j in range(n):
            self.collist[j].sort()
        self.nnz = int(len(ids))

    def count_row_range(self, i: int, clo: int, chi: int) -> int:
        """Entries of row i with column in [clo, chi]."""
        return sum(1 for j in self.rowlist[i] if clo <= j <= chi)


# ---------------------------------------------------------------- band extractor
def fit_ribbon(R: Residual, i: int, d: int, delta: float, w_max: int):
    cols = R.rowlist[i]
    c = i + d
    if c < 0 or c >= R.n or c not in cols:
        return (0, 0, 0)
    p = cols.index(c)
    lo = hi = p
    l = u = 0
    z = 1
    while True:
        cand = []  # (width, side, new_l, new_u)
        if lo > 0 and c - cols[lo - 1] <= w_max:
            nl = c - cols[lo - 1]
            cand.append((nl + u + 1, 0, nl, u))
        if hi + 1 < len(cols) and cols[hi + 1] - c <= w_max:
            nu = cols[hi + 1] - c
            cand.append((l + nu + 1, 1, l, nu))
        if not cand:
            break
        cand.sort()
        width, side, nl, nu = cand[0]
        if (z + 1) / width < delta:
            break
        z += 1
        l, u = nl, nu
        if side == 0:
            lo -= 1
        else:
            hi += 1
    return (l, u, z)


def grow_segments(R: Residual, ext, d: int, delta: float, l_seg: int):
    m = R.m
    S = []
    i = 0
    while i < m:
        if ext[i][2] == 0:
            i += 1
            continue
        i0 = i
        L, U = ext[i][0], ext[i][1]
        z = R.count_row_range(i0, i0 + d - L, i0 + d + U)
        j = i + 1
        while j < m and ext[j][2] > 0:
            L2, U2 = max(L, ext[j][0]), max(U, ext[j][1])
            if L2 != L or U2 != U:
                z2 = sum(R.count_row_range(r, r + d - L2, r + d + U2) for r in range(i0, j + 1))
            else:
                z2 = z + R.count_row_range(j, j + d - L, j + d + U)
            if z2 / ((L2 + U2 + 1) * (j - i0 + 1)) < delta:
                break
            L, U, z = L2, U2, z2
            j += 1
        if j - i0 >= l_seg:
            S.append((i0, j, L, U, z))
        i = j
    return S


def extract_bands(R: Residual, p: Params):
    """Algorithm 3.  Returns segments (row_start, row_end, d, L, U, z) in acceptance order."""
    m, n = R.m, R.n
    d_max = p.d_max if p.d_max > 0 else max(m, n)
    count_min = p.count_min if p.count_min > 0 else int(math.ceil(p.delta * p.l_seg))
    M: Dict[int, int] = {}
    for i in range(m):
        for j in R.rowlist[i]:
            d = j - i
            if abs(d) <= d_max:
                M[d] = M.get(d, 0) + 1
    D = sorted([d for d, c in M.items() if c >= count_min], key=lambda d: (-M[d], d))
    used = [False] * m
    out = []
    for d in D:
        ext = [(0, 0, 0) if used[i] else fit_ribbon(R, i, d, p.delta, p.w_max) for i in range(m)]
        S = grow_segments(R, ext, d, p.delta, p.l_seg)
        if not S:
            continue
        area = sum((L + U + 1) * (j - i0) for (i0, j, L, U, z) in S)
        zz = sum(z for (_, _, _, _, z) in S)
        if area < p.a_min or zz / area < p.delta:
            continue
        for (i0, j, L, U, z) in S:
            for r in range(i0, j):
                used[r] = True
            out.append((i0, j, d, L, U, z))
    return out


# ---------------------------------------------------------------- block extractor
def _isqrt_ceil(a: int) -> int:
    s = math.isqrt(a)
    return s if s * s >= a else s + 1


def score2(nnz: int, a: int, delta: float) -> float:
    """The square of Algorithm 2's score a (d - delta)^1.5, d = nnz / a:
    (nnz - delta a)^3 / a.  It orders windows as the score does (both grow
    with the score for d >= delta) and needs only IEEE multiply, subtract and
    divide, which round alike everywhere, unlike a library pow."""
    t = float(nnz) - delta * float(a)
    if t < 0.0:           # d >= delta by division while the product rounds below
        t = 0.0
    return t * t * t / float(a)


def find_block(lines: List[List[int]], O0: int, O1: int, I0: int, I1: int, p: Params):
    """Algorithm 2 over outer lines [O0, O1) and inner range [I0, I1).

    Returns (score2, o0, o1_end, i0, i1_end) with half-open ends, score2 -1 if
    none; score2 is the square of the printed score (see score2).
    """
    best = (-1.0, 0, 0, 0, 0)
    s_min = _isqrt_ceil(p.a_min)
    L_in = I1 - I0
    for o0 in range(O0, O1):
        H = [0] * L_in
        for o1 in range(o0, min(O1, o0 + p.max_span)):
            for j in lines[o1]:
                if I0 <= j < I1:
                    H[j - I0] += 1
            s = o1 - o0 + 1
            if s < s_min:
                continue
            nnz = 0
            i0 = 0
            for i1 in range(L_in):
                nnz += H[i1]
                while i0 <= i1:
                    a = s * (i1 - i0 + 1)
                    if a < p.a_min:
                        break
                    dens = nnz / a
                    if dens >= p.delta:
                        sc = score2(nnz, a, p.delta)
                        if sc > best[0]:
                            best = (sc, o0, o1 + 1, I0 + i0, I0 + i1 + 1)
                        break
                    nnz -= H[i0]
                    i0 += 1
    return best


def _block_nnz(R: Residual, r0, r1, c0, c1) -> int:
    return sum(R.count_row_range(i, c0, c1 - 1) for i in range(r0, r1))


def trim(R: Residual, r0, r1, c0, c1):
    nnz = _block_nnz(R, r0, r1, c0, c1)
    while True:
        area = (r1 - r0) * (c1 - c0)
        best = None  # (new_nnz, new_area, edge)
        edges = []
        if r1 - r0 >= 2:
            edges.append(("top", R.count_row_range(r0, c0, c1 - 1), c1 - c0))
            edges.append(("bottom", R.count_row_range(r1 - 1, c0, c1 - 1), c1 - c0))
        if c1 - c0 >= 2:
            edges.append(("left", sum(1 for i in R.collist[c0] if r0 <= i < r1), r1 - r0))
            edges.append(("right", sum(1 for i in R.collist[c1 - 1] if r0 <= i < r1), r1 - r0))
        for name, e_nnz, e_len in edges:
            nn, na = nnz - e_nnz, area - e_len
            if nn * area <= nnz * na:          # no strict density gain
                continue
            if best is None or nn * best[1] > best[0] * na:
                best = (nn, na, name)
        if best is None:
            return r0, r1, c0, c1, nnz
        nnz = best[0]
        if best[2] == "top":
            r0 += 1
        elif best[2] == "bottom":
            r1 -= 1
        elif best[2] == "left":
            c0 += 1
        else:
            c1 -= 1


def candidate_regions(R: Residual, p: Params):
    m, n, g = R.m, R.n, p.tile
    TI, TJ = (m + g - 1) // g, (n + g - 1) // g
    cnt: Dict[Tuple[int, int], int] = {}
    for i in range(m):
        for j in R.rowlist[i]:
            key = (i // g, j // g)
            cnt[key] = cnt.get(key, 0) + 1
    hot = set()
    for (I, J), c in cnt.items():
        area = min(g, m - I * g) * min(g, n - J * g)
        if c >= p.delta * area:
            hot.add((I, J))
    seen = set()
    boxes = []
    S = max(1, -(-p.max_span // g))            # slab height in cells
    for t in sorted(hot):
        if t in seen:
            continue
        stack = [t]
        seen.add(t)
        comp = []
        I0, I1, J0, J1 = t[0], t[0] + 1, t[1], t[1] + 1
        while stack:
            a, b = stack.pop()
            comp.append((a, b))
            I0, I1, J0, J1 = min(I0, a), max(I1, a + 1), min(J0, b), max(J1, b + 1)
            for da in (-1, 0, 1):
                for db in (-1, 0, 1):
                    q = (a + da, b + db)
                    if q in hot and q not in seen:
                        seen.add(q)
                        stack.append(q)
        if I1 - I0 > S and 4 * len(comp) < (I1 - I0) * (J1 - J0):
            # a tall component filling under a quarter of its box: one box per slab
            for a in range(I0, I1, S):
                b = min(I1, a + S)
                cols = [c for (r, c) in comp if a <= r < b]
                boxes.append([max(0, a - 1) if a == I0 else a, min(TI, b + 1) if b == I1 else b,
                              max(0, min(cols) - 1), min(TJ, max(cols) + 2)])
        else:
            boxes.append([max(0, I0 - 1), min(TI, I1 + 1), max(0, J0 - 1), min(TJ, J1 + 1)])
    merged = True
    while merged:
        merged = False
        boxes.sort()
        for x in range(len(boxes)):
            for y in range(x + 1, len(boxes)):
                A, B = boxes[x], boxes[y]
                if A[0] < B[1] and B[0] < A[1] and A[2] < B[3] and B[2] < A[3]:
                    boxes[x] = [min(A[0], B[0]), max(A[1], B[1]), min(A[2], B[2]), max(A[3], B[3])]
                    del boxes[y]
                    merged = True
                    break
            if merged:
                break
    boxes.sort()
    return [(I0 * g, min(m, I1 * g), J0 * g, min(n, J1 * g)) for (I0, I1, J0, J1) in boxes]


def partition_blocks(R: Residual, p: Params):
    """Algorithm 1.  Returns accepted blocks (r0, r1, c0, c1, nnz) in acceptance order."""
    used_r = [False] * R.m
    used_c = [False] * R.n
    blocks = []

    def decompose(r0, r1, c0, c1):
        if (r1 - r0) * (c1 - c0) < p.a_min:
            return
        b = find_block(R.rowlist, r0, r1, c0, c1, p)
        bc = find_block(R.collist, c0, c1, r0, r1, p)
        if bc[0] > b[0]:
            b = (bc[0], bc[3], bc[4], bc[1], bc[2])
        if b[0] < 0:
            return
        _, br0, br1, bc0, bc1 = b
        if (br1 - br0) * (bc1 - bc0) < p.a_min:
            return
        if any(used_r[br0:br1]) or any(used_c[bc0:bc1]):
            return
        br0, br1, bc0, bc1, bnnz = trim(R, br0, br1, bc0, bc1)
        area = (br1 - br0) * (bc1 - bc0)
        if bnnz / area < p.delta or area < p.a_min:
            return
        blocks.append((br0, br1, bc0, bc1, bnnz))
        for i in range(br0, br1):
            used_r[i] = True
        for j in range(bc0, bc1):
            used_c[j] = True
        decompose(r0, br0, c0, c1)
        decompose(br1, r1, c0, c1)
        decompose(br0, br1, c0, bc0)
        decompose(br0, br1, bc1, c1)

    regions = [(0, R.m, 0, R.n)] if p.tile <= 0 else candidate_regions(R, p)
    for (r0, r1, c0, c1) in regions:
        decompose(r0, r1, c0, c1)
    blocks = [b for b in blocks if b[3] - b[2] != 1]
    if sum(b[4] for b in blocks) < p.coverage_min * R.nnz:
        return []
    return blocks


# ---------------------------------------------------------------- plan
@dataclass
class Extraction:
    m: int
    n: int
    rows: np.ndarray           # canonical entries
    cols: np.ndarray
    vals: np.ndarray
    owner: np.ndarray          # VDIA / VBR / CSR per canonical entry
    segments: List[Tuple[int, int, int, int]] = field(default_factory=list)  # (r0, nrows, off_lo, ndiag)
    blocks: List[Tuple[int, int, int, int]] = field(default_factory=list)    # (r0, nrows, c0, ncols)


def run_plan(m: int, n: int, row, col, val, extractors: Sequence[Tuple[int, Optional[Params]]]):
    """Run the extractors in order over the residual (Section 3, 'Extract').

    Raises ValueError when the last extractor leaves entries unclaimed.
    """
    rows, cols, vals = canonicalize(m, n, row, col, val)
    owner = np.full(rows.size, -1, dtype=np.int64)
    ex = Extraction(m, n, rows, cols, vals, owner)
    for kind, p in extractors:
        p = p or default_params(kind)
        ids = np.nonzero(owner < 0)[0]
        R = Residual(m, n, rows[ids], cols[ids], ids)
        if kind == CSR:
            owner[ids] = CSR
        elif kind == VDIA:
            for ps in range(p.passes):
                if ps > 0:   # the next pass sees the residual this one left
                    ids = np.nonzero(owner < 0)[0]
                    R = Residual(m, n, rows[ids], cols[ids], ids)
                for (i0, j, d, L, U, z) in extract_bands(R, p):
                    ex.segments.append((i0, j - i0, d - L, L + U + 1))
                    for r in range(i0, j):
                        for c, e in zip(R.rowlist[r], R.rowids[r]):
                            if d - L <= c - r <= d + U:
                                owner[e] = VDIA
        elif kind == VBR:
            for (r0, r1, c0, c1, z) in partition_blocks(R, p):
                ex.blocks.append((r0, r1 - r0, c0, c1 - c0))
                for r in range(r0, r1):
                    for c, e in zip(R.rowlist[r], R.rowids[r]):
                        if c0 <= c < c1:
                            owner[e] = VBR
        else:
            raise ValueError("unknown extractor")
    if np.any(owner < 0):
        raise ValueError("incomplete plan: residual not empty")
    ex.segments.sort()
    ex.blocks.sort()
    return ex


def merge_segments(segments):
    """VDIA segments of several passes, (row_start, nrows, lowest offset,
    ndiags) each, as one segment list with per-segment offset sets: the rows
    are cut at every segment start and end, and each maximal row range that
    the same segments cover becomes (row_start, nrows, sorted union of their
    offsets).  Rows no segment covers are left out."""
    cuts = sorted({r for (r0, nr, _, _) in segments for r in (r0, r0 + nr)})
    out = []
    for a, b in zip(cuts, cuts[1:]):
        offs = sorted({o for (r0, nr, lo, nd) in segments if r0 <= a and b <= r0 + nr for o in range(lo, lo + nd)})
        if not offs:
            continue
        if out and out[-1][0] + out[-1][1] == a and out[-1][2] == tuple(offs):
            out[-1] = (out[-1][0], out[-1][1] + b - a, out[-1][2])   # same set continues
        else:
            out.append((a, b - a, tuple(offs)))
    return out


def check_partition(ex: Extraction, vdia_cells, vbr_cells, csr_entries) -> None:
    """Exact partition check of stored formats against the canonical matrix.

    Each argument maps (i, j) -> stored value for the cells one format holds
    (a format may hold a cell as padding: a cell inside a band or block whose
    entry is absent or was claimed by another format).  Asserts, bit-exactly:
    a canonical entry with value v != 0 is held with value v by exactly one
    format and as 0 by any other; a canonical explicit zero is held by at
    least one format; every CSR entry is canonical; every other held cell
    stores 0.
    """
    canon = {(int(i), int(j)): np.float32(v) for i, j, v in zip(ex.rows, ex.cols, ex.vals)}
    holders: Dict[Tuple[int, int], List[np.float32]] = {}
    for name, cells in (("vdia", vdia_cells), ("vbr", vbr_cells), ("csr", csr_entries)):
        for key, v in cells.items():
            if name == "csr":
                assert key in canon, f"CSR holds non-entry {key}"
            holders.setdefault(key, []).append(np.float32(v))
    for key, vs in holders.items():
        bits = [int(np.float32(v).view(np.uint32)) for v in vs]
        if key in canon:
            cb = int(canon[key].view(np.uint32))
            nonzero = [b for b in bits if b != 0]
            if cb == 0:
                assert not nonzero, f"explicit zero {key} holds a value"
            else:
                assert nonzero == [cb], f"entry {key}: stored {vs}, canonical {canon[key]}"
        else:
            assert all(b == 0 for b in bits), f"padding cell {key} is not +0"
    missing = set(canon) - set(holders)
    assert not missing, f"{len(missing)} entries unclaimed"
