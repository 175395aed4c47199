"""Row-range sharding of a matrix over ranks (one process per GPU).

The hybrid form shards by rows: VDIA segments and VBR blocks are row ranges,
so each rank extracts and runs a plan for its own rows of A, computes its own
rows of y (or C) with no reduction, and needs the whole x (or B), which is
replicated when it is constant or all-gathered otherwise.  Cuts are placed so
that the ranks hold nearly equal numbers of entries."""
from __future__ import annotations

import numpy as np


def row_cuts(m: int, row, world: int) -> np.ndarray:
    """world + 1 row boundaries, 0 = c_0 <= ... <= c_world = m, splitting the
    entries (row indices `row`) as evenly as whole rows allow."""
    if world < 1:
        raise ValueError("world must be >= 1")
    counts = np.bincount(np.asarray(row, dtype=np.int64), minlength=m) if m else np.zeros(0, np.int64)
    csum = np.concatenate([[0], np.cumsum(counts)])
    total = int(csum[-1])
    cuts = [0]
    for r in range(1, world):
        cuts.append(max(cuts[-1], int(np.searchsorted(csum, total * r / world, side="left"))))
    cuts.append(m)
    return np.minimum(np.array(cuts, dtype=np.int64), m)


def shard(A: dict, world: int, rank: int):
    """(row0, row1, sub-matrix dict) of rank's rows; the sub-matrix keeps all n
    columns and renumbers rows from 0."""
    cuts = row_cuts(A["m"], A["row"], world)
    r0, r1 = int(cuts[rank]), int(cuts[rank + 1])
    sel = (A["row"] >= r0) & (A["row"] < r1)
    sub = dict(m=r1 - r0, n=A["n"], row=(A["row"][sel] - r0).astype(np.int32), col=A["col"][sel].astype(np.int32),
               val=A["val"][sel])
    return r0, r1, sub
