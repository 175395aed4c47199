"""Tiling of a batch: the grouped SpMV launch over many plans (sable_batch_*)
runs every plan with its own row tiles, and the grouped SpMM launch uses the
first plan's column panel and depth, so the batch is tuned as a whole.  Each
candidate is set on every plan (SpMV tiles need a new upload), a batch is
built and its grouped launch timed with CUDA events (replayed from a CUDA
graph, as a batch is meant to be run); the fastest candidate is left
applied.  Single plans are tuned by the library's own sable_autotune
(Plan.autotune)."""
from __future__ import annotations

from . import BF16_BLOCKS, FP32, Batch

SPMV_CANDIDATES = [(r, b) for r in (128, 256, 512, 1024) for b in (16 << 10, 48 << 10, 160 << 10)]
SPMM_CANDIDATES = [(c, d) for c in (0, 32, 64, 128) for d in (4, 8)]   # (column panel, B rows in flight)


def _time(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(2):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = t if best is None else min(best, t)
    return best


def tune_batch(plans, op, ins, outs, N=0, reps=10, stream=None):
    """op "spmv" (ins = xs, outs = ys) or "spmm_fp32" / "spmm_bf16" (ins = Bs,
    outs = Cs, N columns).  Returns (best tiling dict, {candidate: ms})."""
    import torch
    stream = stream or torch.cuda.current_stream()
    cur = plans[0].tiling()
    cands = SPMV_CANDIDATES if op == "spmv" else SPMM_CANDIDATES
    times = {}
    for a, b in cands:
        t = dict(cur)
        if op == "spmv":
            t.update(spmv_rows=a, spmv_bytes=b)
        else:
            t.update(spmm_cols=a, spmm_depth=b)
        for P in plans:
            P.set_tiling(**t)
            if op == "spmv":
                P.upload(stream)   # SpMV tiles are tables; the SpMM panel and depth are launch knobs
        B = Batch(plans)
        if op == "spmv":
            g = B.graph_spmv(ins, outs)
        else:
            g = B.graph_spmm(ins, outs, N, FP32 if op == "spmm_fp32" else BF16_BLOCKS)
        times[(a, b)] = _time(lambda: g.launch(stream), reps, stream)
        g.close()
        B.close()
    a, b = min(times, key=times.get)
    best = dict(cur)
    if op == "spmv":
        best.update(spmv_rows=a, spmv_bytes=b)
    else:
        best.update(spmm_cols=a, spmm_depth=b)
    for P in plans:
        P.set_tiling(**best)
        if op == "spmv":
            P.upload(stream)
    return best, times
