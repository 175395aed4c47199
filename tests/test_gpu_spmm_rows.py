"""SpMM through the row-split launch (after the tensor-core launch for BF16
and three-term blocks): rows that several parts cover, rows no part covers,
matrices without a CSR remainder, odd widths and several column panels, and
VBR blocks of two stages that share rows (those stay on the FP32 path in
every precision)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu

PRECS = (sable.FP32, sable.BF16_BLOCKS, sable.FP32_SPLIT)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _spmm(P, Bn, prec):
    C = torch.full((P.m, Bn.shape[1]), float("nan"), device="cuda")
    P.spmm(torch.from_numpy(np.ascontiguousarray(Bn)).cuda(), C, prec)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _shared_rows_matrix(values):
    # two dense blocks on the same rows: the first VBR stage can take only one
    # (blocks of a stage are row-disjoint), the second stage takes the other
    rng = np.random.default_rng(21)
    return synth.assemble(rng, 500, 520, blocks=[(40, 10, 150, 120, 1.0), (40, 300, 150, 130, 1.0)],
                          n_scatter=4000, values=values)


SHARED_PLAN = [(sable.VBR, dict(a_min=400, max_span=200, tile=8)), (sable.VBR, dict(a_min=400, max_span=200, tile=8)),
               (sable.CSR, None)]


@pytest.mark.parametrize("N", [128, 36])
def test_blocks_sharing_rows(N):
    A = _shared_rows_matrix("int")
    P = sable.plan_from(A, SHARED_PLAN)
    blks = P.blocks()
    assert len(blks) == 2 and blks[0][0] == blks[1][0], blks   # same rows, two stages
    Bn = synth.dense_operand(4, A["n"], N, dist="int")
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bn)
    for prec in PRECS:   # integer data: exact on the FP32 path every precision takes here
        np.testing.assert_array_equal(_spmm(P, Bn, prec).astype(np.float64), ref)
    P.close()


def test_blocks_sharing_rows_in_a_batch():
    A1 = _shared_rows_matrix("uniform")
    rng = np.random.default_rng(5)
    A2 = synth.assemble(rng, 400, 400, blocks=[(0, 0, 130, 70, 1.0)], n_scatter=2500)
    P1 = sable.plan_from(A1, SHARED_PLAN)
    P2 = sable.plan_from(A2, [(sable.VBR, dict(a_min=400, max_span=200, tile=8)), (sable.CSR, None)])
    assert P2.info()["n_blocks"] == 1
    N = 64
    Bs = [torch.from_numpy(synth.dense_operand(30 + i, A["n"], N)).cuda() for i, A in enumerate((A1, A2))]
    for prec, tol in ((sable.FP32, 1e-5), (sable.BF16_BLOCKS, 2e-2), (sable.FP32_SPLIT, 1e-5)):
        Cs = [torch.full((A["m"], N), float("nan"), device="cuda") for A in (A1, A2)]
        B = sable.Batch([P1, P2])
        B.spmm(Bs, Cs, N, prec)
        torch.cuda.synchronize()
        for A, Bi, Ci, t in ((A1, Bs[0], Cs[0], 1e-5), (A2, Bs[1], Cs[1], tol)):
            ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bi.cpu().numpy())
            assert oracle.normwise_err(Ci.cpu().numpy(), ref) <= t
        B.close()
    P1.close()
    P2.close()


@pytest.mark.parametrize("N", [128, 200, 20, 7])
def test_no_csr_remainder_and_empty_rows(N):
    """All entries in bands and blocks (no CSR entries): every covered row skips
    the row-split pass; rows no part covers (and empty rows) come out zero."""
    rng = np.random.default_rng(8)
    A = synth.assemble(rng, 700, 650, bands=[(0, 0, 300), (1, 0, 300)],
                       blocks=[(400, 100, 120, 96, 1.0)])
    P = sable.plan_from(A, [(sable.VBR, dict(a_min=400, max_span=200, tile=8)),
                            (sable.VDIA, dict(delta=0.75, a_min=100, l_seg=16)), (sable.CSR, None)])
    info = P.info()
    assert info["nnz_csr"] == 0 and info["n_blocks"] == 1 and info["n_segments"] >= 1
    Bn = synth.dense_operand(6, A["n"], N)
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bn)
    for prec in PRECS:
        C = _spmm(P, Bn, prec)
        assert np.all(C[530:] == 0.0) and np.all(C[300:400] == 0.0)
        assert oracle.normwise_err(C, ref) <= (2e-2 if prec == sable.BF16_BLOCKS else 1e-5)
    P.close()


@pytest.mark.parametrize("cols,depth", [(0, 4), (0, 8), (64, 4), (32, 4)])
@pytest.mark.parametrize("N", [128, 132, 36])
def test_all_three_formats_row_split(N, cols, depth):
    rng = np.random.default_rng(12)
    A = synth.mixed_matrix(rng, 3000, 30.0, side_max=96)
    P = sable.plan_from(A, [(sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16)),
                            (sable.VBR, dict(a_min=256, max_span=256)), (sable.CSR, None)])
    P.set_tiling(**dict(P.tiling(), spmm_cols=cols, spmm_depth=depth))
    P.upload()
    info = P.info()
    assert info["nnz_vdia"] > 0 and info["nnz_vbr"] > 0 and info["nnz_csr"] > 0
    Bn = synth.dense_operand(3, A["n"], N)
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bn)
    for prec in PRECS:
        assert oracle.normwise_err(_spmm(P, Bn, prec), ref) <= (2e-2 if prec == sable.BF16_BLOCKS else 1e-5)
    C = torch.full((A["m"], N), float("nan"), device="cuda")
    P.csr_spmm(torch.from_numpy(Bn).cuda(), C)
    torch.cuda.synchronize()
    assert oracle.normwise_err(C.cpu().numpy(), ref) <= 1e-5
    P.close()


def _mixed_batch_mats():
    rng = np.random.default_rng(31)
    mats = [
        (synth.assemble(rng, 900, 800, n_scatter=6000, values="int"), [(sable.CSR, None)]),   # no per-row list
        (synth.assemble(rng, 1200, 1200, bands=[(o, 0, 1200) for o in (-1, 0, 1)], n_scatter=3000),
         [(sable.VDIA, dict(delta=0.75, a_min=100, l_seg=16)), (sable.CSR, None)]),
        (synth.assemble(rng, 700, 650, blocks=[(100, 30, 140, 90, 1.0)], n_scatter=2000, values="int"),
         [(sable.VBR, dict(a_min=400, max_span=200, tile=8)), (sable.CSR, None)]),
        (_shared_rows_matrix("uniform"), SHARED_PLAN),
        (dict(m=300, n=200, row=np.zeros(0, np.int32), col=np.zeros(0, np.int32), val=np.zeros(0, np.float32)),
         [(sable.CSR, None)]),                                                        # no entries at all
        (synth.assemble(rng, 5, 3000, n_scatter=40), [(sable.CSR, None)]),             # a few long rows
        (synth.mixed_matrix(rng, 2500, 25.0, side_max=96),
         [(sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16)), (sable.VBR, dict(a_min=256, max_span=256)),
          (sable.CSR, None)]),
    ]
    return mats


@pytest.mark.parametrize("N", [32, 64, 20])
def test_batch_mixes_plain_csr_plans_with_structured_ones(N):
    """A batch holding plain-CSR plans (no segments or blocks: no per-row
    structure list), band-only, block-only, two block stages on shared rows,
    a matrix without entries and one with a few very long rows: the grouped
    row-split SpMM (and the block launches before it) against the FP64
    oracle in every precision; integer matrices exactly."""
    mats = _mixed_batch_mats()
    plans = [sable.plan_from(A, spec) for A, spec in mats]
    assert plans[0].info()["n_segments"] == plans[0].info()["n_blocks"] == 0
    assert plans[2].info()["n_blocks"] == 1 and len(plans[3].blocks()) == 2
    ints = {0, 2}
    Bs = [torch.from_numpy(synth.dense_operand(50 + i, A["n"], N, dist="int" if i in ints else "uniform")).cuda()
          for i, (A, _) in enumerate(mats)]
    B = sable.Batch(plans)
    for prec in PRECS:
        Cs = [torch.full((A["m"], N), float("nan"), device="cuda") for A, _ in mats]
        B.spmm(Bs, Cs, N, prec)
        torch.cuda.synchronize()
        for i, ((A, _), Bi, Ci) in enumerate(zip(mats, Bs, Cs)):
            ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bi.cpu().numpy())
            got = Ci.cpu().numpy()
            if i in ints:
                np.testing.assert_array_equal(got.astype(np.float64), ref)
            else:
                tol = 2e-2 if prec == sable.BF16_BLOCKS and plans[i].info()["n_blocks"] else 1e-5
                assert oracle.normwise_err(got, ref) <= tol, (i, prec)
    xs = [torch.from_numpy(synth.dense_operand(70 + i, A["n"])).cuda() for i, (A, _) in enumerate(mats)]
    ys = [torch.full((A["m"],), float("nan"), device="cuda") for A, _ in mats]
    B.spmv(xs, ys)
    torch.cuda.synchronize()
    for (A, _), x, y in zip(mats, xs, ys):
        ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x.cpu().numpy())
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    assert B.device_error() == 0
    B.close()
    for P in plans:
        P.close()


@pytest.mark.parametrize("N", [128, 64, 36, 7])
def test_fp32_blocks_in_row_groups_exact_on_integers(N):
    """FP32 blocks through the row-group block kernel (block rows of C stored
    first) with bands and a CSR remainder on the same rows: integer data, so
    the result equals the FP64 oracle bit for bit; blocks whose heights are
    not multiples of the 8-row group."""
    rng = np.random.default_rng(44)
    A = synth.assemble(rng, 900, 880, bands=[(o, 0, 900) for o in (-1, 0, 1)],
                       blocks=[(13, 200, 53, 77, 1.0), (300, 500, 129, 64, 0.9), (700, 20, 9, 150, 1.0)],
                       n_scatter=5000, values="int")
    P = sable.plan_from(A, [(sable.VBR, dict(a_min=400, max_span=200, tile=8)),
                            (sable.VDIA, dict(delta=0.75, a_min=100, l_seg=16)), (sable.CSR, None)])
    assert P.info()["n_blocks"] >= 2
    Bn = synth.dense_operand(8, A["n"], N, dist="int")
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bn)
    for cols in (0, 64, 32):
        P.set_tiling(**dict(P.tiling(), spmm_cols=cols))   # the panel applies at the next SpMM
        np.testing.assert_array_equal(_spmm(P, Bn, sable.FP32).astype(np.float64), ref)
    P.close()
