"""GPU parity of the batched (grouped, one launch per op) SpMV / SpMM over
many matrices of uneven size, direct and replayed from a CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu

PLAN = [(sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16)), (sable.VBR, dict(a_min=256, max_span=256)),
        (sable.CSR, None)]


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1234)
    mats, plans = [], []
    for k in range(14):
        m = int(np.exp(rng.uniform(np.log(300), np.log(6000))))
        A = synth.mixed_matrix(rng, m, float(np.exp(rng.uniform(np.log(5), np.log(60)))),
                               values="int" if k % 2 else "uniform", side_max=96)
        mats.append(A)
        plans.append(sable.plan_from(A, PLAN))
    kinds = sum(1 for P in plans if P.info()["n_blocks"] > 0)
    assert kinds >= 3, "want several matrices with VBR blocks"
    B = sable.Batch(plans)
    yield mats, plans, B
    B.close()
    for P in plans:
        P.close()


def test_batch_spmv_and_graph(batch):
    mats, plans, B = batch
    xs = [torch.from_numpy(synth.dense_operand(i, A["n"])).cuda() for i, A in enumerate(mats)]
    ys = [torch.full((A["m"],), float("nan"), device="cuda") for A in mats]
    B.spmv(xs, ys)
    torch.cuda.synchronize()
    for A, x, y in zip(mats, xs, ys):
        ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x.cpu().numpy())
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    g = B.graph_spmv(xs, ys)
    for rep in range(2):
        for i, x in enumerate(xs):
            x.copy_(torch.from_numpy(synth.dense_operand(100 + 10 * rep + i, x.numel())))
            ys[i].fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        for A, x, y in zip(mats, xs, ys):
            ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x.cpu().numpy())
            assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    g.close()
    assert B.device_error() == 0


@pytest.mark.parametrize("N", [32, 20])
def test_batch_spmm_fp32_bf16(batch, N):
    mats, plans, B = batch
    Bs = [torch.from_numpy(synth.dense_operand(7 + i, A["n"], N, dist="int" if i % 2 else "uniform")).cuda()
          for i, A in enumerate(mats)]
    for prec in (sable.FP32, sable.BF16_BLOCKS, sable.FP32_SPLIT):
        Cs = [torch.full((A["m"], N), float("nan"), device="cuda") for A in mats]
        B.spmm(Bs, Cs, N, prec)
        torch.cuda.synchronize()
        for i, (A, Bi, Ci) in enumerate(zip(mats, Bs, Cs)):
            ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bi.cpu().numpy())
            got = Ci.cpu().numpy()
            if i % 2:   # integer values and operand: exact in every precision
                np.testing.assert_array_equal(got.astype(np.float64), ref)
            else:
                assert oracle.normwise_err(got, ref) <= (2e-2 if prec == sable.BF16_BLOCKS else 1e-5)
    g = B.graph_spmm(Bs, Cs, N, sable.BF16_BLOCKS)
    for Ci in Cs:
        Ci.fill_(float("nan"))
    g.launch()
    torch.cuda.synchronize()
    for i, (A, Bi, Ci) in enumerate(zip(mats, Bs, Cs)):
        ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bi.cpu().numpy())
        assert oracle.normwise_err(Ci.cpu().numpy(), ref) <= 2e-2
    g.close()


def test_batch_tiling_tuner():
    """tune.tune_batch re-uploads every plan per candidate tiling; the plans it
    leaves behind (the fastest tiling) still compute the right products."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00829_gb300 import tune
    rng = np.random.default_rng(77)
    mats = [synth.mixed_matrix(rng, int(m), 20.0, side_max=96) for m in (800, 2500, 4000, 1200)]
    plans = [sable.plan_from(A, PLAN) for A in mats]
    xs = [torch.from_numpy(synth.dense_operand(i, A["n"])).cuda() for i, A in enumerate(mats)]
    ys = [torch.empty(A["m"], device="cuda") for A in mats]
    best, times = tune.tune_batch(plans, "spmv", xs, ys, reps=3)
    assert (best["spmv_rows"], best["spmv_bytes"]) in times and len(times) == len(tune.SPMV_CANDIDATES)
    N = 16
    Bs = [torch.from_numpy(synth.dense_operand(50 + i, A["n"], N)).cuda() for i, A in enumerate(mats)]
    Cs = [torch.empty(A["m"], N, device="cuda") for A in mats]
    bm, _ = tune.tune_batch(plans, "spmm_bf16", Bs, Cs, N=N, reps=3)
    assert all((P.tiling()["spmm_cols"], P.tiling()["spmm_depth"]) == (bm["spmm_cols"], bm["spmm_depth"])
               for P in plans)
    B = sable.Batch(plans)
    for y in ys:
        y.fill_(float("nan"))
    B.spmv(xs, ys)
    B.spmm(Bs, Cs, N, sable.FP32)
    torch.cuda.synchronize()
    for i, A in enumerate(mats):
        ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs[i].cpu().numpy())
        assert oracle.normwise_err(ys[i].cpu().numpy(), ref) <= 1e-5
        refC = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bs[i].cpu().numpy())
        assert oracle.normwise_err(Cs[i].cpu().numpy(), refC) <= 1e-5
    B.close()
    for P in plans:
        P.close()


def test_empty_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B = sable.Batch([])
    B.spmv([], [])
    B.close()
