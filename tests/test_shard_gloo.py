"""Row sharding over two ranks (gloo, CPU): each rank takes its row range of
the matrix, extracts a library plan of its rows (host extraction: VDIA, VBR
and CSR stages), checks that the plan's three formats hold exactly its rows'
entries, computes its rows of y with the FP64 oracle from those format
arrays, and the all-gathered pieces equal the single-process result
exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_2407_00829_gb300 as sable
from paper_2407_00829_gb300 import shard
import synth


def _plan_entries(P, n):
    """(row, col, val) of the nonzero cells a plan stores in its VDIA, VBR and
    CSR arrays, sorted by (row, col); a cell stored twice fails."""
    cells = {}

    def put(r, c, v):
        assert (r, c) not in cells, (r, c)
        cells[(r, c)] = v

    vals, k = P.vdia_values(), 0
    for (r0, nr, lo, nd) in P.segments().tolist():
        for o in range(lo, lo + nd):
            for r in range(r0, r0 + nr):
                if 0 <= r + o < n and vals[k] != 0:
                    put(r, r + o, vals[k])
                k += 1
    vals, k = P.vbr_values(), 0
    for (r0, nr, c0, nc) in P.blocks().tolist():
        for c in range(c0, c0 + nc):
            for r in range(r0, r0 + nr):
                if vals[k] != 0:
                    put(r, c, vals[k])
                k += 1
    rp, ci, cv = P.csr()
    for r in range(len(rp) - 1):
        for q in range(rp[r], rp[r + 1]):
            put(r, int(ci[q]), cv[q])
    keys = sorted(cells)
    return (np.array([a for a, _ in keys], np.int64), np.array([b for _, b in keys], np.int64),
            np.array([cells[t] for t in keys], np.float32))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = synth.mixed_matrix(np.random.default_rng(31), 3000, 12.0)
        x = synth.dense_operand(7, A["n"]).astype(np.float32)
        r0, r1, sub = shard.shard(A, world, rank)
        P = sable.plan_from(sub, [(sable.VDIA, dict(a_min=64, l_seg=8)), (sable.VBR, dict(a_min=64)),
                                  (sable.CSR, None)], upload=False)
        info = P.info()
        rr, cc, vv = _plan_entries(P, sub["n"])
        P.close()
        o = np.lexsort((sub["col"], sub["row"]))
        assert np.array_equal(rr, sub["row"][o]) and np.array_equal(cc, sub["col"][o])
        assert np.array_equal(vv, sub["val"][o])
        y_part = oracle.spmv(sub["m"], rr, cc, vv, x)
        dist.all_gather_object(stats := [None] * world, (info["nnz_vdia"], info["nnz_vbr"], info["nnz_csr"]))
        sizes = [None] * world
        dist.all_gather_object(sizes, (r0, r1))
        pieces = [torch.zeros(b - a, dtype=torch.float64) for a, b in sizes]
        mine = torch.from_numpy(np.ascontiguousarray(y_part))
        # gloo all_gather wants equal sizes: pad to the largest piece
        L = max(b - a for a, b in sizes)
        padded = [torch.zeros(L, dtype=torch.float64) for _ in sizes]
        buf = torch.zeros(L, dtype=torch.float64)
        buf[:mine.numel()] = mine
        dist.all_gather(padded, buf)
        y = torch.cat([p[:b - a] for p, (a, b) in zip(padded, sizes)]).numpy()
        if rank == 0:
            o = np.lexsort((A["col"], A["row"]))
            full = oracle.spmv(A["m"], A["row"][o], A["col"][o], A["val"][o], x)
            out.put((bool(np.array_equal(y, full)), [b - a for a, b in sizes], int(A["row"].size), stats))
    finally:
        dist.destroy_process_group()


def test_row_cuts_balance_entries():
    rng = np.random.default_rng(0)
    A = synth.mixed_matrix(rng, 5000, 20.0)
    for world in (1, 2, 3, 8):
        c = shard.row_cuts(A["m"], A["row"], world)
        assert c[0] == 0 and c[-1] == A["m"] and np.all(np.diff(c) >= 0)
        per = np.diff(np.searchsorted(np.sort(A["row"]), c))
        assert per.sum() == A["row"].size
        assert per.max() - per.min() <= 2 * np.bincount(A["row"]).max() + 1   # each cut within one row of ideal
    assert list(shard.row_cuts(0, np.zeros(0, np.int32), 2)) == [0, 0, 0]


def test_two_rank_row_shards_concat_to_the_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    equal, sizes, nnz, stats = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert equal and sum(sizes) == 3000 and min(sizes) > 0
    assert sum(map(sum, stats)) == nnz
    assert all(v > 0 and b > 0 for v, b, _ in stats)      # each rank's plan has bands and blocks
