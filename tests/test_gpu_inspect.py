"""Device inspector (the extractors' counting steps on the GPU): the regions,
stored values and CSR remainder equal the host inspector's entry for entry,
and the oracle's on matrices it extracts in seconds.  Integer and index work,
so every comparison is exact.  Cases: the paper-shaped workloads, multi-pass
bands, density floors whose FP64 tests sit on exact ties (0.1, 1/3, 0.6, 0.7),
pre-pass tiles from 1 to 64 with ragged edges, w_max 0 and 512, d_max limits,
empty and one-row matrices."""
import numpy as np
import pytest

import paper_2407_00829_gb300 as sable
import synth
from oracle import extract as ox

pytestmark = pytest.mark.gpu


def _pair(A, spec):
    H = sable.plan_from(A, spec, upload=False)
    D = sable.plan_from(A, spec, upload=False, inspector=sable.INSPECT_DEVICE)
    return H, D


def _same(H, D):
    assert np.array_equal(H.segments(), D.segments())
    assert np.array_equal(H.blocks(), D.blocks())
    assert np.array_equal(H.region_stages()[0], D.region_stages()[0])
    assert np.array_equal(H.region_stages()[1], D.region_stages()[1])
    assert np.array_equal(H.vdia_values(), D.vdia_values())
    assert np.array_equal(H.vbr_values(), D.vbr_values())
    for a, b in zip(H.csr(), D.csr()):
        assert np.array_equal(a, b)
    assert H.info() == D.info()


def _oracle_regions(A, spec):
    ps = []
    for kind, kw in spec:
        p = ox.default_params(kind)
        for k, v in (kw or {}).items():
            setattr(p, k, v)
        ps.append((kind, p))
    ex = ox.run_plan(A["m"], A["n"], A["row"], A["col"], A["val"], ps)
    return sorted(ex.segments), sorted(ex.blocks), int(np.sum(ex.owner == ox.CSR))


def _check(A, spec, oracle=False):
    H, D = _pair(A, spec)
    _same(H, D)
    if oracle:
        segs, blks, ncsr = _oracle_regions(A, spec)
        assert sorted(map(tuple, D.segments().tolist())) == segs
        assert sorted(map(tuple, D.blocks().tolist())) == blks
        assert D.info()["nnz_csr"] == ncsr
    out = D.info()
    H.close()
    D.close()
    return out


def test_blocks_bands_scatter_4096_matches_host_and_oracle():
    A = synth.blocks_bands_scatter_4096()
    info = _check(A, [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)], oracle=True)
    assert info["n_segments"] > 0 and info["n_blocks"] > 0


def test_bands_powerlaw_1m_matches_host():
    A = synth.bands_powerlaw_1m()
    info = _check(A, [(sable.VDIA, None), (sable.CSR, None)])
    assert info["nnz_vdia"] == 3962256
    info = _check(A, [(sable.VDIA, dict(passes=3)), (sable.CSR, None)])
    assert info["nnz_csr"] < 7370556


@pytest.mark.parametrize("passes", [1, 2])
def test_multi_pass_bands_match_oracle(passes):
    rng = np.random.default_rng(11)
    m = 3000
    A = synth.assemble(rng, m, m, bands=[(o, int(rng.integers(0, 800)), int(rng.integers(1500, 2200)))
                                         for o in (-2, -1, 0, 1, 2, -300, -299, 300, 301)], n_scatter=4000)
    _check(A, [(sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16, passes=passes)), (sable.CSR, None)],
           oracle=True)


@pytest.mark.parametrize("delta", [0.1, 1.0 / 3.0, 0.6, 0.7, 1.0])
def test_density_floors_on_exact_ties(delta):
    """Bands with gaps every few cells put (z + 1) / w exactly on small
    fractions such as 1/3 and 3/5, where the FP64 quotient equals the FP64
    delta: the device thresholds must take the host's side of each tie."""
    rng = np.random.default_rng(int(delta * 1000))
    m, n = 1500, 1600
    bands = []
    for o in (-3, -1, 0, 2, 5, 9):
        bands.append((o, int(rng.integers(0, 200)), int(rng.integers(800, 1300))))
    A = synth.assemble(rng, m, n, bands=bands, n_scatter=3000)
    keep = (A["row"] + A["col"]) % 5 != 0          # periodic holes: ribbons of 4 in 5, 2 in 3, ...
    keep |= (A["col"] - A["row"]) == 0
    B = dict(m=m, n=n, row=A["row"][keep], col=A["col"][keep], val=A["val"][keep])
    for w_max in (0, 3, 64, 512):
        _check(B, [(sable.VDIA, dict(delta=delta, a_min=64, l_seg=4, w_max=w_max, count_min=1)),
                   (sable.CSR, None)], oracle=(w_max == 3))


@pytest.mark.parametrize("tile", [1, 3, 8, 64])
def test_block_prepass_tiles_with_ragged_edges(tile):
    rng = np.random.default_rng(100 + tile)
    m, n = 2003, 1997                                   # no tile size divides either
    blocks = [(int(r), int(c), int(s), int(s), 0.8) for r, c, s in
              ((5, 7, 60), (400, 1200, 90), (1900, 1900, 97), (1200, 50, 70))]
    A = synth.assemble(rng, m, n, blocks=blocks, n_scatter=20000)
    spec = [(sable.VBR, dict(delta=0.5, a_min=400, tile=tile)), (sable.CSR, None)]
    info = _check(A, spec, oracle=(tile in (3, 8)))
    assert info["n_blocks"] >= 3


def test_blocks_scatter_200k_matches_host():
    A = synth.blocks_scatter_200k()
    info = _check(A, [(sable.VBR, dict(a_min=256)), (sable.CSR, None)])
    assert info["n_blocks"] > 500


def test_d_max_and_mixed_stage_orders():
    rng = np.random.default_rng(7)
    A = synth.mixed_matrix(rng, 5000, 12.0)
    for spec in ([(sable.VDIA, dict(d_max=3)), (sable.VBR, None), (sable.CSR, None)],
                 [(sable.VBR, dict(tile=4)), (sable.VDIA, dict(delta=0.5)), (sable.CSR, None)],
                 [(sable.VDIA, dict(d_max=1000, passes=2)), (sable.VBR, dict(tile=16)), (sable.CSR, None)]):
        _check(A, spec)


def test_empty_and_degenerate_matrices():
    spec = [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)]
    for m, n in [(0, 0), (5, 0), (0, 7), (6, 6), (1, 1000), (1000, 1)]:
        A = dict(m=m, n=n, row=np.zeros(0, np.int64), col=np.zeros(0, np.int64), val=np.zeros(0, np.float32))
        _check(A, spec)
    rng = np.random.default_rng(5)
    one_row = dict(m=1, n=5000, row=np.zeros(3000, np.int64), col=rng.permutation(5000)[:3000],
                   val=rng.standard_normal(3000).astype(np.float32))
    _check(one_row, spec, oracle=True)
    one_col = dict(m=5000, n=1, row=rng.permutation(5000)[:3000], col=np.zeros(3000, np.int64),
                   val=rng.standard_normal(3000).astype(np.float32))
    _check(one_col, spec, oracle=True)
    dense = synth.assemble(rng, 200, 200, blocks=[(0, 0, 200, 200, 1.0)])
    _check(dense, spec, oracle=True)


def test_device_inspected_plan_computes_like_the_host_one():
    """The plan built by the device inspector runs like the host one: both
    SpMVs match the FP64 oracle within the FP32 bound (the kernels' shared
    atomics make the summation order, not the plan, vary between runs)."""
    import torch
    import oracle
    A = synth.blocks_bands_scatter_4096()
    spec = [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)]
    H = sable.plan_from(A, spec)
    D = sable.plan_from(A, spec, inspector=sable.INSPECT_DEVICE)
    x_np = synth.dense_operand(11, A["n"])
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x_np)
    x = torch.from_numpy(x_np).cuda()
    for P in (H, D):
        y = torch.empty(A["m"], device="cuda")
        P.spmv(x, y)
        torch.cuda.synchronize()
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    H.close()
    D.close()


def test_device_inspector_allocation_failures_return_oom_and_free_memory():
    """Allocation-failure injection at each guarded allocation of a device
    extraction (plan tables on the host, the residual's device copy, the
    histogram, ribbon and cell-key buffers): the extraction returns
    SABLE_ERR_OOM and keeps it as the plan's status, or succeeds with the host
    inspector's plan once the countdown passes every allocation; device memory
    is back where it started."""
    import torch
    L = sable.lib()
    A = synth.blocks_bands_scatter_4096()
    spec = [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)]
    H = sable.plan_from(A, spec, upload=False)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outcomes = []
    try:
        for k in range(12):
            P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
            for kind, kw in spec:
                P.add_extractor(kind, **(kw or {}))
            P.set_inspector(sable.INSPECT_DEVICE)
            L.sable_debug_fail_allocations(k)
            st = L.sable_extract(P.handle)
            L.sable_debug_fail_allocations(-1)
            outcomes.append(st)
            if st == 0:
                _same(H, P)
            else:
                assert st == 2 and L.sable_plan_status(P.handle) == 2
            P.close()
    finally:
        L.sable_debug_fail_allocations(-1)
    assert 2 in outcomes and outcomes[-1] == 0          # some allocation failed; late enough, none does
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    H.close()
