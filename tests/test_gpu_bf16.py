"""GPU parity of SpMM with VBR blocks on the tensor cores: BF16 blocks, and
FP32-accurate blocks as three bf16 terms (SABLE_FP32_SPLIT).

* Integer inputs: block values / s_b and B are exact in bfloat16 and every
  partial sum is an integer below 2^24, so the result must equal the FP64
  oracle bit for bit.  This pins the tensor-core operand layouts.
* Random inputs: against a quantisation-aware FP64 oracle (blocks rounded to
  bf16 of a / s_b times s_b, their B rows rounded to bf16, everything else
  exact; the oracle's own extraction gives the blocks) within 1e-5, and
  against the plain FP64 oracle within the 2e-2 BF16 budget (normwise).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import extract as ox
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu

TOL_Q = 1e-5
TOL_BF16 = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _spmm(P, B, prec):
    C = torch.full((P.m, B.shape[1]), float("nan"), device="cuda")
    P.spmm(torch.from_numpy(np.ascontiguousarray(B)).cuda(), C, prec)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _matrix(seed, values):
    rng = np.random.default_rng(seed)
    m, n = 420, 390
    blocks = [(10, 20, 140, 75, 1.0),      # two 128-row tiles, two K steps (64 + 11)
              (200, 150, 60, 130, 0.85),   # three K steps
              (300, 300, 40, 40, 1.0)]
    return synth.assemble(rng, m, n, blocks=blocks, n_scatter=3000, values=values)


PLAN = [(sable.VBR, dict(a_min=400, max_span=160, tile=8)), (sable.CSR, None)]


@pytest.mark.parametrize("cols,depth", [(0, 4), (64, 4), (128, 8)])
@pytest.mark.parametrize("N", [128, 32, 200])
def test_bf16_integer_exact(N, cols, depth):
    A = _matrix(3, "int")
    P = sable.plan_from(A, PLAN)
    P.set_tiling(**dict(P.tiling(), spmm_cols=cols, spmm_depth=depth))
    assert P.info()["n_blocks"] == 3
    B = synth.dense_operand(5, A["n"], N, dist="int")
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    np.testing.assert_array_equal(_spmm(P, B, sable.BF16_BLOCKS).astype(np.float64), ref)
    P.close()


@pytest.mark.parametrize("N", [128, 64, 250])
def test_bf16_random_vs_quantisation_aware_oracle(N):
    A = _matrix(7, "uniform")
    P = sable.plan_from(A, PLAN)
    ex = ox.run_plan(A["m"], A["n"], A["row"], A["col"], A["val"],
                     [(ox.VBR, ox.Params(delta=0.5, a_min=400, max_span=160, tile=8)), (ox.CSR, None)])
    assert sorted(map(tuple, P.blocks().tolist())) == sorted(ex.blocks)
    B = synth.dense_operand(9, A["n"], N)
    C = _spmm(P, B, sable.BF16_BLOCKS)
    # quantisation-aware reference from the oracle's blocks
    inb = ex.owner == ox.VBR
    qv = ex.vals.copy()
    for (r0, nr, c0, nc) in ex.blocks:
        sel = inb & (ex.rows >= r0) & (ex.rows < r0 + nr) & (ex.cols >= c0) & (ex.cols < c0 + nc)
        s = oracle.pow2_scale(float(np.max(np.abs(ex.vals[sel]))) if sel.any() else 0.0)
        qv[sel] = oracle.bf16_round(ex.vals[sel] / np.float32(s)) * np.float32(s)
    ref_q = (oracle.spmm(A["m"], ex.rows[inb], ex.cols[inb], qv[inb], oracle.bf16_round(B)) +
             oracle.spmm(A["m"], ex.rows[~inb], ex.cols[~inb], ex.vals[~inb], B))
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    assert oracle.normwise_err(C, ref_q) <= TOL_Q
    assert oracle.normwise_err(C, ref) <= TOL_BF16
    # the FP32 path on the same plan stays at FP32 accuracy
    assert oracle.normwise_err(_spmm(P, B, sable.FP32), ref) <= 1e-5
    P.close()


def test_bf16_without_blocks_equals_fp32():
    rng = np.random.default_rng(1)
    A = synth.assemble(rng, 300, 300, n_scatter=2000)
    P = sable.plan_from(A, PLAN)
    assert P.info()["n_blocks"] == 0
    B = synth.dense_operand(2, 300, 16)
    np.testing.assert_array_equal(_spmm(P, B, sable.BF16_BLOCKS), _spmm(P, B, sable.FP32))
    P.close()


@pytest.mark.parametrize("N", [128, 32, 200])
def test_fp32_split_integer_exact(N):
    A = _matrix(3, "int")
    P = sable.plan_from(A, PLAN)
    B = synth.dense_operand(5, A["n"], N, dist="int")
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    np.testing.assert_array_equal(_spmm(P, B, sable.FP32_SPLIT).astype(np.float64), ref)
    P.close()


@pytest.mark.parametrize("N", [128, 64, 250])
def test_fp32_split_within_fp32_tolerance(N):
    """Three-term blocks on the tensor cores meet the FP32 budget (1e-5
    normwise against FP64), with inputs of mixed magnitude."""
    A = _matrix(7, "normal")
    A["val"] = (A["val"] * np.exp(np.random.default_rng(1).uniform(-6, 6, A["val"].size))).astype(np.float32)
    P = sable.plan_from(A, PLAN)
    assert P.info()["n_blocks"] == 3
    B = synth.dense_operand(9, A["n"], N, dist="normal")
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    err_split = oracle.normwise_err(_spmm(P, B, sable.FP32_SPLIT), ref)
    err_bf16 = oracle.normwise_err(_spmm(P, B, sable.BF16_BLOCKS), ref)
    assert err_split <= 1e-5
    assert err_split < err_bf16 / 50       # three terms, not one
    P.close()
