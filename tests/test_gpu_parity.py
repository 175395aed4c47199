"""GPU parity: the library's CUDA SpMV/SpMM (through the C ABI) against the FP64
oracle on the same seeded inputs.  Tolerance: normwise relative error
||y - y_ref||_inf / ||y_ref||_inf <= 1e-5 for FP32; bit-exact on integer
inputs whose partial sums stay below 2^24 (every FP32 rounding is exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
ALL3 = [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _spmv(P, x, plain=False):
    y = torch.full((P.m,), float("nan"), device="cuda")
    (P.csr_spmv if plain else P.spmv)(_dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _spmm(P, B, plain=False, precision=sable.FP32):
    C = torch.full((P.m, B.shape[1]), float("nan"), device="cuda")
    if plain:
        P.csr_spmm(_dev(B), C)
    else:
        P.spmm(_dev(B), C, precision)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _small_cases():
    out = []
    for seed in range(6):
        rng = np.random.default_rng(700 + seed)
        m = int(rng.integers(300, 2500))
        n = int(rng.integers(300, 2500))
        bands = [(o, int(rng.integers(0, m // 3)), int(rng.integers(m // 3, m))) for o in (-1, 0, 1)]
        bands.append((int(rng.integers(-n // 2, n // 2)), 0, m))
        blocks = []
        if min(m, n) > 400:
            blocks = [(int(rng.integers(0, m - 150)), int(rng.integers(0, n - 150)), 60, 70, 0.9)]
        A = synth.assemble(rng, m, n, bands=bands, blocks=blocks,
                           row_lengths=synth.powerlaw_lengths(rng, m, kmax=300))
        out.append(A)
    return out


SMALL = _small_cases()
PLANS = [
    [(sable.VDIA, dict(delta=0.75, a_min=200, l_seg=16)), (sable.VBR, dict(a_min=400, max_span=128)),
     (sable.CSR, None)],
    [(sable.VDIA, dict(delta=0.75, a_min=200, l_seg=16)), (sable.CSR, None)],
    [(sable.VBR, dict(a_min=400, max_span=128)), (sable.CSR, None)],
    [(sable.CSR, None)],
]


@pytest.mark.parametrize("case", range(len(SMALL)))
@pytest.mark.parametrize("plan", range(len(PLANS)))
def test_spmv_small(case, plan):
    A = SMALL[case]
    P = sable.plan_from(A, PLANS[plan])
    x = synth.dense_operand(case, A["n"])
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)
    assert oracle.normwise_err(_spmv(P, x), ref) <= TOL_FP32
    assert oracle.normwise_err(_spmv(P, x, plain=True), ref) <= TOL_FP32
    P.close()


@pytest.mark.parametrize("tiling", [dict(spmv_rows=4, spmv_bytes=64, spmm_cols=32),
                                    dict(spmv_rows=1024, spmv_bytes=1 << 22, spmm_depth=8),
                                    dict(spmv_rows=36, spmv_bytes=300, spmm_cols=64)])
def test_spmv_integer_exact_any_tiling(tiling):
    rng = np.random.default_rng(42)
    m, n = 1501, 1203
    A = synth.assemble(rng, m, n, bands=[(o, 3, 1400) for o in (-2, -1, 0, 1, 2)] + [(700, 0, 1500)],
                       blocks=[(400, 800, 100, 90, 0.85)], row_lengths=synth.powerlaw_lengths(rng, m, kmax=200),
                       values="int")
    P = sable.plan_from(A, [(sable.VDIA, dict(a_min=100, l_seg=8)), (sable.VBR, dict(a_min=400)),
                            (sable.CSR, None)], tiling=tiling)
    info = P.info()
    assert info["nnz_vdia"] > 0 and info["nnz_vbr"] > 0 and info["nnz_csr"] > 0
    x = synth.dense_operand(3, n, dist="int")
    ref = oracle.spmv(m, A["row"], A["col"], A["val"], x)
    np.testing.assert_array_equal(_spmv(P, x).astype(np.float64), ref)
    B = synth.dense_operand(4, n, 12, dist="int")
    refC = oracle.spmm(m, A["row"], A["col"], A["val"], B)
    np.testing.assert_array_equal(_spmm(P, B).astype(np.float64), refC)
    P.close()


def test_spmv_x_not_16_byte_aligned():
    """x starting 4 bytes past an aligned address takes the scalar load path."""
    A = SMALL[1]
    P = sable.plan_from(A, ALL3)
    xs = synth.dense_operand(21, A["n"])
    buf = torch.zeros(A["n"] + 1, device="cuda")
    buf[1:] = torch.from_numpy(xs).cuda()
    x = buf[1:]
    assert x.data_ptr() % 16 != 0
    y = torch.full((A["m"],), float("nan"), device="cuda")
    P.spmv(x, y)
    torch.cuda.synchronize()
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs)
    assert oracle.normwise_err(y.cpu().numpy(), ref) <= TOL_FP32
    P.close()


def test_edge_cases():
    # empty matrix, zero rows/cols, a single very long row, an all-empty tail
    cases = [dict(m=10, n=7, row=np.zeros(0, np.int32), col=np.zeros(0, np.int32), val=np.zeros(0, np.float32)),
             dict(m=1, n=5000, row=np.zeros(5000, np.int32), col=np.arange(5000, dtype=np.int32),
                  val=np.linspace(-1, 1, 5000).astype(np.float32)),
             dict(m=3000, n=3, row=np.arange(3000, dtype=np.int32) % 7, col=np.arange(3000, dtype=np.int32) % 3,
                  val=np.ones(3000, np.float32))]
    for A in cases:
        P = sable.plan_from(A, ALL3)
        x = synth.dense_operand(1, A["n"])
        ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)
        y = _spmv(P, x)
        if np.abs(ref).max() == 0:
            assert np.all(y == 0)
        else:
            assert oracle.normwise_err(y, ref) <= TOL_FP32
        P.close()
    P = sable.plan_from(dict(m=0, n=4, row=[], col=[], val=[]), ALL3)
    P.spmv(torch.zeros(4, device="cuda"), torch.zeros(0, device="cuda"))
    P.close()


def test_order_errors_on_device():
    P = sable.Plan(4, 4, [0], [0], [1.0]).add_extractor(sable.CSR).extract()
    with pytest.raises(sable.SableError) as e:
        P.spmv(torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda"))
    assert e.value.status == 5
    P.upload()
    with pytest.raises(sable.SableError) as e:
        P.spmm(torch.zeros(4, 0, device="cuda"), torch.zeros(4, 0, device="cuda"))
    assert e.value.status == 1
    P.close()


@pytest.mark.parametrize("cols,depth", [(0, 4), (64, 4), (32, 4), (128, 8)])
@pytest.mark.parametrize("N", [1, 7, 32, 128, 200])
def test_spmm_small(N, cols, depth):
    A = SMALL[2]
    P = sable.plan_from(A, PLANS[0])
    P.set_tiling(**dict(P.tiling(), spmm_cols=cols, spmm_depth=depth))
    B = synth.dense_operand(N, A["n"], N)
    ref = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    assert oracle.normwise_err(_spmm(P, B), ref) <= TOL_FP32
    assert oracle.normwise_err(_spmm(P, B, plain=True), ref) <= TOL_FP32
    P.close()


def test_blocks_bands_scatter_4096():
    A = synth.blocks_bands_scatter_4096()
    P = sable.plan_from(A, ALL3)
    info = P.info()
    assert info["n_blocks"] == 8 and info["n_segments"] >= 1
    x = synth.dense_operand(11, A["n"])
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)
    assert oracle.normwise_err(_spmv(P, x), ref) <= TOL_FP32
    B = synth.dense_operand(12, A["n"], 128)
    refC = oracle.spmm(A["m"], A["row"], A["col"], A["val"], B)
    assert oracle.normwise_err(_spmm(P, B), refC) <= TOL_FP32
    P.close()


@pytest.mark.slow
def test_bands_powerlaw_1m_full_size():
    A = synth.bands_powerlaw_1m()
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.CSR, None)])
    x = synth.dense_operand(7, A["n"], dist="normal")
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)
    assert oracle.normwise_err(_spmv(P, x), ref) <= TOL_FP32
    assert oracle.normwise_err(_spmv(P, x, plain=True), ref) <= TOL_FP32
    P.close()


@pytest.mark.slow
def test_blocks_scatter_200k_full_size_sampled():
    """Full-size SpMM (200k^2, ~30M entries, N=128) in FP32 and with BF16
    blocks, checked on 3000 sampled rows of C against the FP64 oracle."""
    A = synth.blocks_scatter_200k()
    P = sable.plan_from(A, [(sable.VBR, dict(a_min=256)), (sable.CSR, None)])
    assert P.info()["n_blocks"] > 700
    B = synth.dense_operand(13, A["n"], 128)
    sel = np.random.default_rng(0).choice(A["m"], 3000, replace=False)
    ref = oracle.spmm_rows(A["m"], A["row"], A["col"], A["val"], B, sel)
    Bd = _dev(B)
    for cols, depth in ((0, 4), (64, 4), (128, 8)):
        P.set_tiling(**dict(P.tiling(), spmm_cols=cols, spmm_depth=depth))
        for prec, tol in ((sable.FP32, TOL_FP32), (sable.BF16_BLOCKS, 2e-2), (sable.FP32_SPLIT, TOL_FP32)):
            C = torch.empty(A["m"], 128, device="cuda")
            P.spmm(Bd, C, prec)
            torch.cuda.synchronize()
            assert oracle.normwise_err(C[torch.from_numpy(sel).cuda()].cpu().numpy(), ref) <= tol
    P.close()


def test_single_plan_calls_replay_from_a_cuda_graph():
    """SpMV (hybrid and plain CSR) and SpMM (FP32 blocks) of one plan captured
    in a CUDA graph on a side stream and replayed twice, with new x / B
    values copied in between: every replay matches the oracle."""
    A = synth.blocks_bands_scatter_4096()
    P = sable.plan_from(A, ALL3)
    m, n, N = A["m"], A["n"], 64
    x = torch.empty(n, device="cuda")
    y = torch.empty(m, device="cuda")
    yp = torch.empty(m, device="cuda")
    B = torch.empty(n, N, device="cuda")
    C = torch.empty(m, N, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        P.spmv(x, y, side)
        P.csr_spmv(x, yp, side)
        P.spmm(B, C, sable.FP32, side)
    for seed in (21, 22):
        xs = synth.dense_operand(seed, n)
        Bs = synth.dense_operand(seed + 100, n, N)
        x.copy_(_dev(xs))
        B.copy_(_dev(Bs))
        y.fill_(float("nan"))
        yp.fill_(float("nan"))
        C.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref = oracle.spmv(m, A["row"], A["col"], A["val"], xs)
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= TOL_FP32
        assert oracle.normwise_err(yp.cpu().numpy(), ref) <= TOL_FP32
        refC = oracle.spmm(m, A["row"], A["col"], A["val"], Bs)
        assert oracle.normwise_err(C.cpu().numpy(), refC) <= TOL_FP32
    del g
    P.close()


def test_long_rows_cut_across_tiles():
    """Rows of 150,000 entries (two in one 4-row group, one alone) among short
    rows: their tiles' CSR ranges are cut into chunks summed by other CTAs,
    and a second launch adds the partial sums.  Hybrid and plain CSR SpMV
    match the oracle on repeated calls and under CUDA-graph replay; a batch
    refuses the plan (its grouped launch has no second launch)."""
    rng = np.random.default_rng(61)
    m = n = 200_000
    long_rows = (10, 11, 50_003)
    R = [rng.integers(0, m, 1_000_000)]
    C = [rng.integers(0, n, 1_000_000)]
    for r in long_rows:
        cols = rng.choice(n, 150_000, replace=False)
        R.append(np.full(cols.size, r))
        C.append(cols)
    i = np.arange(m)
    R.append(i)
    C.append(i)
    row = np.concatenate(R)
    col = np.concatenate(C)
    key = np.unique(row * n + col)
    A = dict(m=m, n=n, row=(key // n).astype(np.int32), col=(key % n).astype(np.int32),
             val=rng.uniform(-1, 1, key.size).astype(np.float32))
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.CSR, None)])
    x = synth.dense_operand(62, n)
    ref = oracle.spmv(m, A["row"], A["col"], A["val"], x)
    for _ in range(3):
        assert oracle.normwise_err(_spmv(P, x), ref) <= TOL_FP32
        assert oracle.normwise_err(_spmv(P, x, plain=True), ref) <= TOL_FP32
    xd = _dev(x)
    y = torch.empty(m, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        P.spmv(xd, y, side)
    for _ in range(2):
        y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= TOL_FP32
    del g
    with pytest.raises(sable.SableError) as e:
        sable.Batch([P])
    assert e.value.status == 8
    P.close()
