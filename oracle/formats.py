"""Reference layouts of the two structured formats, built from a given partition.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* VDIA (Section 4.2.1, Fig. 4): segments are contiguous row ranges, each with
  its own list of diagonal offsets.  ``val`` is diagonal-major inside a
  segment: for every offset of the segment, the values of all its rows in
  row order.  Per segment: starting row, row count, diagonal count, start in
  ``val`` and start in ``idiag``.
* VBR (Appendix B, Fig. 9): SPARSKIT's variable block row format.  ``Rpntr``
  and ``Cpntr`` cut rows and columns into block rows/columns; ``Bpntrb`` is a
  CSR-style pointer into ``Bindx`` (block-column index of each stored block);
  ``Indx`` gives the start of each block inside ``Val``, with a final entry
  equal to ``len(Val)``; each block is stored column-major.

Matrices are passed as a dict {(i, j): value} holding the structural entries.
Cells inside a segment or block with no entry are stored as 0.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

Entries = Dict[Tuple[int, int], float]


def vdia_arrays(entries: Entries, ncols: int,
                segments: Sequence[Tuple[int, int, Sequence[int]]]):
    """Pack VDIA arrays.

    ``segments`` lists (row_start, nrows, offsets) in the order they are to be
    stored.  A cell (r, r + off) outside [0, ncols) is stored as 0.
    """
    val: List[float] = []
    idiag: List[int] = []
    seg_row_start, seg_nrows, seg_ndiags, seg_val_ptr, seg_idiag_ptr = [], [], [], [], []
    for (r0, nr, offs) in segments:
        seg_row_start.append(r0)
        seg_nrows.append(nr)
        seg_ndiags.append(len(offs))
        seg_val_ptr.append(len(val))
        seg_idiag_ptr.append(len(idiag))
        for off in offs:
            idiag.append(int(off))
            for r in range(r0, r0 + nr):
                c = r + off
                val.append(entries.get((r, c), 0.0) if 0 <= c < ncols else 0.0)
    return dict(val=val, idiag=idiag, seg_row_start=seg_row_start, seg_nrows=seg_nrows,
                seg_ndiags=seg_ndiags, seg_val_ptr=seg_val_ptr, seg_idiag_ptr=seg_idiag_ptr)


def vbr_arrays(entries: Entries, rpntr: Sequence[int], cpntr: Sequence[int],
               stored: Sequence[Tuple[int, int]]):
    """Pack SPARSKIT VBR arrays.

    ``stored`` lists the (block row, block column) pairs that are kept as
    dense blocks; they are emitted block row by block row, in increasing
    block-column order inside a block row.
    """
    by_row: Dict[int, List[int]] = {}
    for (bi, bj) in stored:
        by_row.setdefault(bi, []).append(bj)
    nbrows = len(rpntr) - 1
    val: List[float] = []
    indx: List[int] = []
    bindx: List[int] = []
    bpntrb: List[int] = [0]
    for bi in range(nbrows):
        for bj in sorted(by_row.get(bi, [])):
            indx.append(len(val))
            bindx.append(bj)
            for c in range(cpntr[bj], cpntr[bj + 1]):          # column-major block
                for r in range(rpntr[bi], rpntr[bi + 1]):
                    val.append(entries.get((r, c), 0.0))
        bpntrb.append(len(bindx))
    indx.append(len(val))
    return dict(Val=val, Indx=indx, Bindx=bindx, Rpntr=list(rpntr), Cpntr=list(cpntr),
                Bpntrb=bpntrb)


def block_values_colmajor(entries: Entries, r0: int, nr: int, c0: int, nc: int) -> List[float]:
    """Values of one dense block [r0, r0+nr) x [c0, c0+nc), column-major, fill 0."""
    return [entries.get((r, c), 0.0) for c in range(c0, c0 + nc) for r in range(r0, r0 + nr)]
