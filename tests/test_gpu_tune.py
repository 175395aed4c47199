"""Autotuner: the chosen tiling is one of the candidates, the plan computes
the same result with it, and the choice is remembered per shape class."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu

SPMV_ROWS, SPMV_BYTES = {32, 64, 128, 256, 512, 1024}, {4 << 10, 16 << 10, 48 << 10, 160 << 10}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_autotune_spmv_and_spmm():
    sable.autotune_cache_clear()
    A = synth.mixed_matrix(np.random.default_rng(8), 30_000, 24.0)
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.VBR, dict(a_min=256)), (sable.CSR, None)])
    xs = synth.dense_operand(1, A["n"])
    x, y = torch.from_numpy(xs).cuda(), torch.empty(A["m"], device="cuda")
    t, ms = P.autotune(sable.TUNE_SPMV, x, y, reps=5)
    # a fixed candidate, or 1024 rows with a wave-sized byte target
    assert (t["spmv_rows"] in SPMV_ROWS and t["spmv_bytes"] in SPMV_BYTES) or t["spmv_rows"] == 1024
    assert ms > 0
    assert P.tiling() == t
    y.fill_(float("nan"))
    P.spmv(x, y)
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs)
    assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    Bs = synth.dense_operand(2, A["n"], 64)
    B, C = torch.from_numpy(Bs).cuda(), torch.empty(A["m"], 64, device="cuda")
    refm = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bs)
    for op, tol in ((sable.TUNE_SPMM_FP32, 1e-5), (sable.TUNE_SPMM_BF16, 2e-2)):
        tm, msm = P.autotune(op, B, C, reps=3)
        assert (tm["spmm_cols"], tm["spmm_depth"]) in ((128, 4), (128, 8), (64, 4), (64, 8), (32, 4), (32, 8))
        assert msm > 0
        assert (tm["spmv_rows"], tm["spmv_bytes"]) == (t["spmv_rows"], t["spmv_bytes"])   # SpMV choice kept
        C.fill_(float("nan"))
        P.spmm(B, C, sable.FP32 if op == sable.TUNE_SPMM_FP32 else sable.BF16_BLOCKS)
        assert oracle.normwise_err(C.cpu().numpy(), refm) <= tol
    # a second plan of the same shape class reuses the remembered SpMV tiling
    Q = sable.plan_from(A, [(sable.VDIA, None), (sable.VBR, dict(a_min=256)), (sable.CSR, None)])
    t2, _ = Q.autotune(sable.TUNE_SPMV, x, y, reps=5)
    assert (t2["spmv_rows"], t2["spmv_bytes"]) == (t["spmv_rows"], t["spmv_bytes"])
    assert sable.autotune_cache_clear() == 3
    P.close()
    Q.close()


def test_autotune_plain_csr():
    """The plain-CSR comparison path has its own tuner op; the tiling it picks
    keeps both the plain and the hybrid SpMV correct."""
    sable.autotune_cache_clear()
    A = synth.mixed_matrix(np.random.default_rng(9), 20_000, 18.0)
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.CSR, None)])
    xs = synth.dense_operand(3, A["n"])
    x, y = torch.from_numpy(xs).cuda(), torch.empty(A["m"], device="cuda")
    t, ms = P.autotune(sable.TUNE_CSR_SPMV, x, y, reps=5)
    assert (t["spmv_rows"] in SPMV_ROWS and t["spmv_bytes"] in SPMV_BYTES) or t["spmv_rows"] == 1024
    assert ms > 0 and P.tiling() == t
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs)
    for fn in (P.csr_spmv, P.spmv):
        y.fill_(float("nan"))
        fn(x, y)
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    assert sable.autotune_cache_clear() == 1
    P.close()
