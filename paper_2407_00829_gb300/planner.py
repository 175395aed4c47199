"""Plan selection: the exhaustive planner and a learned one.

A plan is an ordered list of extractors with their thresholds: the paper's
knobs are the extractor order (Section 4.3), the block threshold delta and
A_min (Section 4.1) and the band threshold delta (Section 5 uses 0.75).  The
exhaustive planner extracts, uploads and times every candidate plan on the
device and keeps the fastest; it is the fallback and the yardstick.  The learned
planner computes the matrix's structural features with the library's feature
kernels, asks a small MLP (trained by the library's own forward / backward /
Adam kernels on timings the pipeline produced) for every candidate's
predicted slowdown log(t / t_best), and extracts only the predicted best plan.

Data set work flow (matrices from ``synth.planner_set_matrix``):

  regions  (host only)  extract every candidate plan of matrices [start, stop)
                        and save their region tables, one .npz per matrix
  collect  (device)     rebuild each candidate plan from its region table (or
                        extract it when no table is given), time SpMV and
                        SpMM (N = 64, BF16 blocks) with CUDA events, compute
                        the device features; write features + timings
  evaluate (device)     train on the first matrices, score on the held-out
                        rest: plan-quality loss t_chosen / t_exhaustive - 1
  select   (device)     as evaluate, after choosing the ensemble size, steps
                        and learning rate on a validation part of the
                        training matrices
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import os
import time
import zlib

import numpy as np

from . import (BF16_BLOCKS, CSR, NFEAT, VBR, VDIA, Mlp, Plan, features, load_region_table,
               save_region_table)

CANDIDATES = [
    ("csr", [(CSR, None)]),
    ("vdia0.6+csr", [(VDIA, dict(delta=0.6)), (CSR, None)]),
    ("vdia0.75+csr", [(VDIA, dict(delta=0.75)), (CSR, None)]),
    ("vdia0.9+csr", [(VDIA, dict(delta=0.9)), (CSR, None)]),
    ("vbr0.5+csr", [(VBR, dict(delta=0.5, a_min=256)), (CSR, None)]),
    ("vbr0.7+csr", [(VBR, dict(delta=0.7, a_min=256)), (CSR, None)]),
    ("vdia0.75+vbr0.5+csr", [(VDIA, dict(delta=0.75)), (VBR, dict(delta=0.5, a_min=256)), (CSR, None)]),
    ("vdia0.75+vbr0.7+csr", [(VDIA, dict(delta=0.75)), (VBR, dict(delta=0.7, a_min=256)), (CSR, None)]),
    ("vbr0.5+vdia0.75+csr", [(VBR, dict(delta=0.5, a_min=256)), (VDIA, dict(delta=0.75)), (CSR, None)]),
]
NAMES = [c[0] for c in CANDIDATES]
DEFAULT = "vdia0.75+vbr0.5+csr"       # the three-format composition at the paper's thresholds
OPS = [("spmv", 0), ("spmm64_bf16", 64)]
N_IN = NFEAT + 1                       # structural features + the product's N


def op_feature(N: int) -> float:
    return math.log2(N + 1.0) / 8.0


def checksum(A) -> int:
    """CRC of the structure (extraction depends on the structure only)."""
    c = zlib.crc32(np.ascontiguousarray(A["row"], np.int32).tobytes())
    return zlib.crc32(np.ascontiguousarray(A["col"], np.int32).tobytes(), c)


def _new_plan(A) -> Plan:
    return Plan(A["m"], A["n"], A["row"], A["col"], A["val"])


def _extract(A, spec, inspector: int = 0) -> Plan:
    P = _new_plan(A)
    for kind, kw in spec:
        P.add_extractor(kind, **(kw or {}))
    if inspector:
        P.set_inspector(inspector)
    return P.extract()


# ---------------------------------------------------------------- host: tables
def region_tables(A, candidates=CANDIDATES):
    """Extract every candidate plan; return {name: region table}."""
    out = {}
    for name, spec in candidates:
        P = _extract(A, spec)
        out[name] = P.region_table()
        P.close()
    return out


def save_matrix_tables(path, A, tables):
    arrs = {"checksum": np.array([checksum(A)], np.int64), "shape": np.array([A["m"], A["n"], A["row"].size])}
    for c, name in enumerate(NAMES):
        for t, (kind, g) in enumerate(tables[name]):
            arrs[f"c{c}_s{t}_k{kind}"] = np.asarray(g, np.int32)
    np.savez_compressed(path, **arrs)


def load_matrix_tables(path):
    d = np.load(path)
    tables = {}
    for c, name in enumerate(NAMES):
        st = sorted((k for k in d.files if k.startswith(f"c{c}_s")), key=lambda k: int(k.split("_")[1][1:]))
        tables[name] = [(int(k.split("_k")[1]), d[k].astype(np.int64)) for k in st]
    return tables, int(d["checksum"][0])


# ---------------------------------------------------------------- device: timing
def matrix_features(A, device="cuda") -> np.ndarray:
    import torch
    row = torch.from_numpy(np.ascontiguousarray(A["row"], dtype=np.int32)).to(device)
    col = torch.from_numpy(np.ascontiguousarray(A["col"], dtype=np.int32)).to(device)
    return features(A["m"], A["n"], row, col).cpu().numpy()


def _time_ms(fn, warm=3, rounds=5, min_ms=1.5, reps=None):
    """Mean device ms of one launch over back-to-back launches, best of
    `rounds`; each round runs enough launches to last about min_ms (events
    around each launch would also time the host's launch gaps, a large and
    noisy share of a tens-of-microseconds SpMV, and short rounds leave the
    minimum noisy)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(warm):
        fn()
    b.record()
    torch.cuda.synchronize()
    if reps is None:
        est = max(a.elapsed_time(b) / warm, 1e-3)
        reps = int(min(2000, max(10, math.ceil(min_ms / est))))
    best = float("inf")
    for _ in range(rounds):
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / reps)
    return best


def _op_fn(P, N, x, y, B, C):
    return (lambda: P.spmv(x, y)) if N == 0 else (lambda: P.spmm(B, C, BF16_BLOCKS))


def time_plan(P, A, x, y, B, C, rounds=5):
    """Device ms of each op in OPS for one uploaded plan."""
    return [_time_ms(_op_fn(P, N, x, y, B, C), rounds=rounds) for _, N in OPS]


def time_candidates(plans, A, x, y, B, C, top=3):
    """ms of every candidate x op; the `top` fastest of each op are then timed
    again with twice the rounds and keep their best, so that the exhaustive
    planner's minimum is not a noise low of one candidate."""
    t = np.array([time_plan(P, A, x, y, B, C) for P in plans], np.float64)
    for o, (_, N) in enumerate(OPS):
        for c in np.argsort(t[:, o])[:top]:
            t[c, o] = min(t[c, o], _time_ms(_op_fn(plans[c], N, x, y, B, C), rounds=10))
    return t


def build_plans(A, tables=None, workers=9, upload=True, inspector: int = 0):
    """All candidate plans of A (uploaded unless upload=False): from region
    tables when given; searched with the host inspector, or with the device
    inspector (INSPECT_DEVICE: the same plans)."""
    def one(c):
        name, spec = CANDIDATES[c]
        if tables is None:
            return _extract(A, spec, inspector)
        return _new_plan(A).add_stages(tables[name]).extract()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        plans = list(ex.map(one, range(len(CANDIDATES))))
    if upload:
        for P in plans:
            P.upload()
    return plans


def _operands(A, seed):
    import torch
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.standard_normal(A["n"]).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((A["n"], OPS[1][1])).astype(np.float32)).cuda()
    y = torch.empty(A["m"], device="cuda")
    C = torch.empty(A["m"], OPS[1][1], device="cuda")
    return x, y, B, C


def exhaustive(A, op=0, tables=None, inspector: int = 0):
    """The exhaustive planner: (best candidate index, ms per candidate, seconds)."""
    t0 = time.perf_counter()
    plans = build_plans(A, tables, inspector=inspector)
    x, y, B, C = _operands(A, 0)
    t = [time_plan(P, A, x, y, B, C)[op] for P in plans]
    for P in plans:
        P.close()
    return int(np.argmin(t)), t, time.perf_counter() - t0


def collect(indices, seed=1005, rows=(100_000, 1_000_000), table_dir=None, log=None, ahead=3):
    """Features and timings (candidates x ops) of the given planner matrices.
    Host threads generate the next `ahead` matrices and rebuild their
    candidate plans while the device times the current one."""
    import synth

    def prepare(i):
        A = synth.planner_set_matrix(i, seed=seed, rows=rows)
        tables, from_tables = None, 0
        if table_dir:
            tables, crc = load_matrix_tables(os.path.join(table_dir, f"m{i:05d}.npz"))
            if crc == checksum(A):
                from_tables = 1
            else:   # another structure than the tables were made for: extract here
                tables = None
        return A, build_plans(A, tables, upload=False), from_tables

    feats, times, meta = [], [], []
    indices = list(indices)
    pool = cf.ThreadPoolExecutor(max_workers=ahead)
    futs = [pool.submit(prepare, i) for i in indices[:ahead]]
    for k, i in enumerate(indices):
        A, plans, from_tables = futs[k].result()
        futs[k] = None
        if k + ahead < len(indices):
            futs.append(pool.submit(prepare, indices[k + ahead]))
        f = matrix_features(A)
        for P in plans:
            P.upload()
        x, y, B, C = _operands(A, i)
        t = time_candidates(plans, A, x, y, B, C).tolist()
        for P in plans:
            P.close()
        feats.append(f)
        times.append(t)
        meta.append([i, A["m"], A["row"].size, from_tables])
        if log:
            best = [NAMES[int(np.argmin([r[o] for r in t]))] for o in range(len(OPS))]
            log(f"{i} m={A['m']} nnz={A['row'].size} tables={from_tables} best={best}")
    return dict(features=np.array(feats, np.float32), times=np.array(times, np.float64),
                meta=np.array(meta, np.int64), names=np.array(NAMES), ops=np.array([o for o, _ in OPS]))


# ---------------------------------------------------------------- learning
def design(data):
    """Rows (matrix, op): inputs [features, op feature], targets log(t / t_best)."""
    F, T = data["features"], data["times"]          # T: [matrices, candidates, ops]
    X, Y = [], []
    for i in range(F.shape[0]):
        for o, (_, N) in enumerate(OPS):
            t = T[i, :, o]
            X.append(np.concatenate([F[i], [op_feature(N)]]))
            Y.append(np.log(t / t.min()))
    return np.array(X, np.float32), np.array(Y, np.float32)


class LearnedPlanner:
    """An ensemble of MLPs N_IN -> h -> h -> len(NAMES) on the library's
    kernels; the prediction is the members' mean (members differ only in
    their seeded initialisation)."""

    def __init__(self, hidden=64, seed=0, members=5):
        self.nets = [Mlp(N_IN, hidden, hidden, len(NAMES), seed=seed + k) for k in range(members)]

    def fit(self, X, Y, steps=2000, lr=2e-3):
        import torch
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
        losses = []
        for net in self.nets:
            for s in range(steps):
                loss = net.grad(Xd, Yd)
                net.adam(lr=lr)
            losses.append(float(loss.item()))
        return losses

    def predict(self, X):
        import torch
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        return np.mean([net.forward(Xd).cpu().numpy() for net in self.nets], axis=0)

    def choose(self, X):
        return np.argmin(self.predict(X), axis=1)

    def plan(self, A, N=0):
        """The learned planner: the chosen candidate's name for matrix A."""
        x = np.concatenate([matrix_features(A), [op_feature(N)]])[None, :]
        return NAMES[int(self.choose(x)[0])]

    def save(self, path, **extra):
        with open(path, "w") as f:
            json.dump(dict(extra, names=NAMES, n_in=N_IN, hidden=self.nets[0].shape.n_h1,
                           params=[[float(v) for v in net.params.cpu().numpy()] for net in self.nets]), f)

    @classmethod
    def load(cls, path):
        import torch
        with open(path) as f:
            d = json.load(f)
        if d["names"] != NAMES or d["n_in"] != N_IN:
            raise ValueError("weights were trained for another candidate set")
        lp = cls(hidden=d["hidden"], members=len(d["params"]))
        for net, p in zip(lp.nets, d["params"]):
            net.params.copy_(torch.tensor(p, dtype=torch.float32))
        return lp


def quality(times, picks):
    """Per (matrix, op): t_pick / t_best - 1; picks is [matrices, ops]."""
    M, _, O = times.shape
    return np.array([[times[i, picks[i, o], o] / times[i, :, o].min() - 1 for o in range(O)] for i in range(M)])


def evaluate(data, n_test=200, steps=2000, seed=0, lp=None, members=5, lr=2e-3):
    """Train on all but the last n_test matrices (unless a trained planner is
    given) and compare on those: the learned planner, the fixed default plan,
    CSR only and the best single candidate on the training matrices."""
    X, Y = design(data)
    n_ops = len(OPS)
    M = data["features"].shape[0]
    cut = M - n_test
    res = {"train_matrices": int(cut), "test_matrices": int(n_test)}
    if lp is None:
        lp = LearnedPlanner(seed=seed, members=members)
        res["train_mse"] = float(np.mean(lp.fit(X[:cut * n_ops], Y[:cut * n_ops], steps=steps, lr=lr)))
    T = data["times"]
    test = T[cut:]
    learned = lp.choose(X[cut * n_ops:]).reshape(n_test, n_ops)
    fixed_best = np.argmin(np.exp(Y[:cut * n_ops]).reshape(cut, n_ops, -1).mean(0), axis=1)   # per op
    picks = {"learned": learned,
             "default": np.full((n_test, n_ops), NAMES.index(DEFAULT)),
             "csr": np.zeros((n_test, n_ops), np.int64),
             "best_fixed": np.tile(fixed_best, (n_test, 1))}
    for k, pk in picks.items():
        q = quality(test, pk)
        res[k] = {op: {"mean_loss": float(q[:, o].mean()), "p90_loss": float(np.quantile(q[:, o], 0.9)),
                       "exact": float(np.mean(q[:, o] == 0))} for o, (op, _) in enumerate(OPS)}
    res["best_fixed_names"] = [NAMES[int(c)] for c in fixed_best]
    # total time of the test set under each planner vs exhaustive
    for k, pk in picks.items():
        res[k]["time_ratio"] = {op: float(sum(test[i, pk[i, o], o] for i in range(n_test)) /
                                          test[:, :, o].min(1).sum()) for o, (op, _) in enumerate(OPS)}
    return res, lp


GRID = [dict(members=m, steps=st, lr=lr) for m in (5, 9) for st in (2000, 4000) for lr in (1e-3, 2e-3)]


def select(data, n_test=200, n_val=80, seed=0, grid=GRID):
    """Model selection without the held-out matrices: each setting is trained
    on the training matrices but the last n_val and scored on those (mean
    plan-quality loss over the ops); the best setting is then trained on all
    training matrices and evaluated once on the held-out n_test."""
    X, Y = design(data)
    n_ops = len(OPS)
    M = data["features"].shape[0]
    cut = M - n_test
    fit_n = cut - n_val
    T = data["times"]
    scores = []
    for g in grid:
        lp = LearnedPlanner(seed=seed, members=g["members"])
        lp.fit(X[:fit_n * n_ops], Y[:fit_n * n_ops], steps=g["steps"], lr=g["lr"])
        picks = lp.choose(X[fit_n * n_ops:cut * n_ops]).reshape(n_val, n_ops)
        scores.append(float(quality(T[fit_n:cut], picks).mean()))
    best = grid[int(np.argmin(scores))]
    res, lp = evaluate(data, n_test=n_test, seed=seed, **best)
    res["selection"] = {"validation_matrices": n_val, "grid": grid, "validation_loss": scores, "chosen": best}
    return res, lp


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["regions", "collect", "evaluate", "select"])
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--stop", type=int, default=600)
    ap.add_argument("--seed", type=int, default=1005)
    ap.add_argument("--tables", default=None, help="directory of region tables")
    ap.add_argument("--out", default="planner_data.npz")
    ap.add_argument("--data", nargs="*", default=[])
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--rows-max", type=int, default=1_000_000,
                    help="matrices' rows drawn log-uniform in [100k, rows-max] (regions and collect alike)")
    a = ap.parse_args()
    rows = (100_000, a.rows_max)
    if a.cmd == "regions":
        import synth
        os.makedirs(a.out, exist_ok=True)
        for i in range(a.start, a.stop):
            path = os.path.join(a.out, f"m{i:05d}.npz")
            if os.path.exists(path):
                continue
            t0 = time.perf_counter()
            A = synth.planner_set_matrix(i, seed=a.seed, rows=rows)
            save_matrix_tables(path + ".tmp.npz", A, region_tables(A))
            os.replace(path + ".tmp.npz", path)
            print(f"{i} m={A['m']} nnz={A['row'].size} {time.perf_counter() - t0:.1f}s", flush=True)
        return
    import torch
    torch.cuda.set_device(0)
    if a.cmd == "collect":
        d = collect(range(a.start, a.stop), seed=a.seed, rows=rows, table_dir=a.tables,
                    log=lambda s: print(s, flush=True))
        np.savez_compressed(a.out, **d)
    else:
        parts = [dict(np.load(p)) for p in a.data]
        d = {k: np.concatenate([p[k] for p in parts]) for k in ("features", "times", "meta")}
        order = np.argsort(d["meta"][:, 0], kind="stable")
        d = {k: v[order] for k, v in d.items()}
        res, lp = select(d, n_test=a.test) if a.cmd == "select" else evaluate(d, n_test=a.test, steps=a.steps)
        print(json.dumps(res))
        if a.out.endswith(".npz"):
            np.savez_compressed(a.out, names=np.array(NAMES), ops=np.array([o for o, _ in OPS]), **d)
        if a.weights:
            lp.save(a.weights, eval=res, data_matrices=int(d["features"].shape[0]))


if __name__ == "__main__":
    main()
