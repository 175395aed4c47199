"""Row sharding over two ranks (gloo, CPU): each rank takes its row range of
the matrix, computes its rows of y with the FP64 oracle, and the all-gathered
pieces equal the single-process result exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2407_00829_gb300 import shard
import synth


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
        y_part = oracle.spmv(sub["m"], sub["row"], sub["col"], sub["val"], x)
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
            full = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)
            out.put((bool(np.array_equal(y, full)), [b - a for a, b in sizes], int(A["row"].size)))
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
    equal, sizes, nnz = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert equal and sum(sizes) == 3000 and min(sizes) > 0
