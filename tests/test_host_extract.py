"""Host logic of the library (no GPU needed): the C ABI loads and exports every
declared symbol, plan rules map to status codes, and the library's C++
extractors produce exactly the oracle's segments, blocks, stored values and
CSR remainder."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import extract as ox
import paper_2407_00829_gb300 as sable
import synth
from conftest import ROOT, read_golden


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "sable.h")).read()
    declared = set(re.findall(r"\b(sable_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    L = sable.lib()
    missing = [d for d in sorted(declared) if not hasattr(L, d)]
    assert not missing, missing
    assert set(sable.EXPORTED) <= declared


def _to_ox_params(kind, kw):
    p = ox.default_params(kind)
    for k, v in (kw or {}).items():
        setattr(p, k, v)
    return p


def _compare(A, extractors):
    """Run the same plan through the library and the oracle; compare exactly."""
    P = sable.plan_from(A, extractors, upload=False)
    ex = ox.run_plan(A["m"], A["n"], A["row"], A["col"], A["val"],
                     [(k, _to_ox_params(k, kw)) for k, kw in extractors])
    segs = sorted(map(tuple, P.segments().tolist()))
    blks = sorted(map(tuple, P.blocks().tolist()))
    assert segs == sorted(ex.segments)
    assert blks == sorted(ex.blocks)
    info = P.info()
    assert info["nnz"] == ex.rows.size
    assert info["nnz_vdia"] == int(np.sum(ex.owner == ox.VDIA))
    assert info["nnz_vbr"] == int(np.sum(ex.owner == ox.VBR))
    assert info["nnz_csr"] == int(np.sum(ex.owner == ox.CSR))
    # stored values, through the exact partition checker
    vd, vb, cs = {}, {}, {}
    vals = P.vdia_values()
    k = 0
    for (r0, nr, lo, nd) in P.segments().tolist():
        for o in range(lo, lo + nd):
            for r in range(r0, r0 + nr):
                if 0 <= r + o < A["n"]:
                    vd[(r, r + o)] = vals[k]
                else:
                    assert vals[k] == 0
                k += 1
    vals = P.vbr_values()
    k = 0
    for (r0, nr, c0, nc) in P.blocks().tolist():
        for c in range(c0, c0 + nc):
            for r in range(r0, r0 + nr):
                vb[(r, c)] = vals[k]
                k += 1
    rp, ci, cv = P.csr()
    for i in range(A["m"]):
        for q in range(rp[i], rp[i + 1]):
            assert (i, int(ci[q])) not in cs
            cs[(i, int(ci[q]))] = cv[q]
        assert list(ci[rp[i]:rp[i + 1]]) == sorted(ci[rp[i]:rp[i + 1]])
    ox.check_partition(ex, vd, vb, cs)
    P.close()
    return ex


def test_fig4_through_the_library():
    g = read_golden("vdia_fig4.txt")
    M = np.array(g["matrix"])
    r, c = np.nonzero(M)
    A = dict(m=10, n=10, row=r, col=c, val=M[r, c].astype(np.float32))
    P = sable.plan_from(A, [(sable.VDIA, dict(delta=0.75, a_min=12, l_seg=3, count_min=3)),
                            (sable.CSR, None)], upload=False)
    assert P.segments().tolist() == [[1, 4, -1, 3], [6, 3, -6, 4]]
    assert P.vdia_values().tolist() == g["val"]
    assert P.info()["nnz_csr"] == 0


@pytest.mark.parametrize("seed", range(4))
def test_three_formats_match_oracle(seed):
    rng = np.random.default_rng(400 + seed)
    m = 180
    bands = [(o, int(rng.integers(0, 40)), int(rng.integers(80, 140))) for o in (-1, 0, 1, 2)]
    bands.append((int(rng.integers(20, 60)), 0, 150))
    blocks = [(120, 10, 30, 24, 0.85), (10, 130, 28, 30, 0.9), (60, 70, 20, 20, 0.7)]
    A = synth.assemble(rng, m, m, bands=bands, blocks=blocks, n_scatter=500)
    _compare(A, [(sable.VDIA, dict(delta=0.75, a_min=200, l_seg=16)),
                 (sable.VBR, dict(delta=0.5, a_min=200, max_span=64, tile=8)),
                 (sable.CSR, None)])


@pytest.mark.parametrize("seed", range(3))
def test_block_partitioner_literal_whole_matrix(seed):
    rng = np.random.default_rng(500 + seed)
    A = synth.assemble(rng, 70, 64, blocks=[(5, 3, 18, 20, 0.9), (40, 30, 20, 25, 0.8)],
                       n_scatter=150)
    _compare(A, [(sable.VBR, dict(delta=0.5, a_min=150, max_span=70, tile=0)), (sable.CSR, None)])


def test_vbr_before_vdia_order():
    rng = np.random.default_rng(9)
    A = synth.assemble(rng, 150, 150, bands=[(o, 0, 150) for o in (-1, 0, 1)],
                       blocks=[(40, 40, 30, 30, 0.95)], n_scatter=200)
    ex = _compare(A, [(sable.VBR, dict(a_min=300, max_span=64)),
                      (sable.VDIA, dict(delta=0.75, a_min=100, l_seg=8)), (sable.CSR, None)])
    assert ex.blocks and ex.segments


@pytest.mark.parametrize("seed", range(2))
def test_band_component_cut_into_slabs(seed):
    """Blocks searched before bands: a 12-diagonal band is a chain of hot
    cells as tall as the matrix; its candidate boxes are slabs of max_span
    rows, and the library and the oracle agree on the result exactly."""
    rng = np.random.default_rng(700 + seed)
    m = 640
    A = synth.assemble(rng, m, m, bands=[(o, 0, m) for o in range(-6, 6)],
                       blocks=[(100, 420, 40, 48, 0.9), (300, 330, 32, 32, 0.95)], n_scatter=800)
    p = ox.Params(delta=0.5, a_min=200, max_span=64, tile=8)
    rows, cols, vals = ox.canonicalize(m, m, A["row"], A["col"], A["val"])
    boxes = ox.candidate_regions(ox.Residual(m, m, rows, cols, np.arange(rows.size)), p)
    tall = [b for b in boxes if b[1] - b[0] > 64 + 16]
    assert not tall, tall                       # every box spans at most one slab (+1 cell each end)
    assert len(boxes) >= m // 64
    ex = _compare(A, [(sable.VBR, dict(delta=0.5, a_min=200, max_span=64, tile=8)),
                      (sable.VDIA, dict(delta=0.75, a_min=200, l_seg=16)), (sable.CSR, None)])
    assert ex.blocks


def test_duplicates_and_explicit_zeros():
    row = np.array([0, 0, 1, 1, 2, 2, 2], np.int32)
    col = np.array([1, 1, 0, 2, 2, 2, 0], np.int32)
    val = np.array([0.5, 0.25, 0.0, 1.0, 1e8, 1.0, -3.0], np.float32)
    A = dict(m=3, n=3, row=row, col=col, val=val)
    P = sable.plan_from(A, [(sable.CSR, None)], upload=False)
    rp, ci, cv = P.csr()
    assert rp.tolist() == [0, 1, 3, 5]
    assert ci.tolist() == [1, 0, 2, 0, 2]
    assert cv.tolist() == [0.75, 0.0, 1.0, -3.0, np.float32(1e8 + 1.0)]
    rows, cols, vals = ox.canonicalize(3, 3, row, col, val)
    assert vals.tolist() == cv[np.lexsort((ci, np.repeat(np.arange(3), np.diff(rp))))].tolist()


def test_status_codes():
    L = sable.lib()
    with pytest.raises(sable.SableError) as e:
        sable.Plan(3, 3, [0, 5], [0, 0], [1.0, 2.0])           # row out of range
    assert e.value.status == 1
    with pytest.raises(sable.SableError) as e:
        sable.Plan(-1, 3, [], [], [])
    assert e.value.status == 1
    P = sable.Plan(4, 4, [0, 1], [0, 3], [1.0, 2.0])
    with pytest.raises(sable.SableError) as e:
        P.info()                                                # before extract
    assert e.value.status == 5
    P.add_extractor(sable.VDIA)
    with pytest.raises(sable.SableError) as e:
        P.extract()                                             # no catch-all extractor
    assert e.value.status == 4
    assert P.status() == 4                                      # sticky
    P.close()
    P = sable.Plan(4, 4, [0], [0], [1.0])
    with pytest.raises(sable.SableError) as e:
        P.add_extractor(sable.VBR, delta=0.0)
    assert e.value.status == 1
    P.add_extractor(sable.CSR).extract()
    with pytest.raises(sable.SableError) as e:
        P.add_extractor(sable.CSR)                              # after extract
    assert e.value.status == 5
    with pytest.raises(sable.SableError) as e:
        P.extract()
    assert e.value.status == 5
    P.close()
    assert L.sable_status_string(4) == b"incomplete plan: entries left unclaimed"


def test_empty_matrix_plans():
    for m, n in [(0, 0), (5, 0), (0, 7), (6, 6)]:
        P = sable.plan_from(dict(m=m, n=n, row=np.zeros(0), col=np.zeros(0), val=np.zeros(0)),
                            [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)], upload=False)
        info = P.info()
        assert info["nnz"] == 0 and info["n_segments"] == 0 and info["n_blocks"] == 0
        P.close()


@pytest.mark.parametrize("seed", range(3))
def test_library_recovers_separated_planted_blocks(seed):
    """Ground truth, not the oracle: full blocks far apart in a sparse matrix
    come back from the library's block extractor (with the candidate-region
    pre-pass) exactly as planted, and so does a short wide block that only the
    column-outer search of Algorithm 1 can find."""
    rng = np.random.default_rng(400 + seed)
    planted = [(4, 6, 20, 24), (60, 70, 30, 18), (120, 120, 25, 30)]
    A = synth.assemble(rng, 160, 160, blocks=[(r0, c0, nr, nc, 1.0) for (r0, c0, nr, nc) in planted],
                       n_scatter=150)
    P = sable.plan_from(A, [(sable.VBR, dict(a_min=300, max_span=64, tile=8)), (sable.CSR, None)], upload=False)
    assert sorted(map(tuple, P.blocks().tolist())) == sorted((r0, nr, c0, nc) for (r0, c0, nr, nc) in planted)
    P.close()
    r, c = np.nonzero(np.pad(np.ones((4, 60)), ((20, 26), (15, 15))))
    A = dict(m=50, n=90, row=r, col=c, val=np.ones(r.size, dtype=np.float32))
    for tile in (0, 8):
        P = sable.plan_from(A, [(sable.VBR, dict(a_min=100, max_span=64, tile=tile)), (sable.CSR, None)],
                            upload=False)
        assert P.blocks().tolist() == [[20, 4, 15, 60]]
        P.close()


def test_wait_limit_bounds_checked_on_the_host():
    L = sable.lib()
    old = sable.wait_limit()
    assert L.sable_set_wait_limit(10) == 1 and L.sable_set_wait_limit(1 << 41) == 1   # SABLE_ERR_INVALID
    assert sable.wait_limit() == old
    sable.set_wait_limit(123456)
    assert sable.wait_limit() == 123456
    sable.set_wait_limit(old)


def test_injected_allocation_failures_return_oom():
    """Host-side allocation-failure injection: the failing call returns
    SABLE_ERR_OOM, a plan that failed keeps it as its status, and the library
    works normally once injection is off."""
    L = sable.lib()
    rng = np.random.default_rng(3)
    A = synth.assemble(rng, 300, 300, bands=[(0, 0, 300), (1, 0, 300)], n_scatter=500)
    row = np.ascontiguousarray(A["row"], np.int32)
    col = np.ascontiguousarray(A["col"], np.int32)
    val = np.ascontiguousarray(A["val"], np.float32)
    import ctypes
    h = ctypes.c_void_p()
    try:
        L.sable_debug_fail_allocations(0)          # the next guarded allocation fails: plan creation
        st = L.sable_plan_create(300, 300, row.size, row.ctypes.data, col.ctypes.data, val.ctypes.data,
                                 ctypes.byref(h))
        assert st == 2 and not h.value             # SABLE_ERR_OOM, no plan handed out
        L.sable_debug_fail_allocations(0)          # creation passes after the reset below
        L.sable_debug_fail_allocations(-1)
        P = sable.Plan(300, 300, row, col, val)
        P.add_extractor(sable.VDIA, a_min=50, l_seg=8).add_extractor(sable.CSR)
        L.sable_debug_fail_allocations(0)          # now extraction's allocation fails
        assert L.sable_extract(P.handle) == 2
        assert L.sable_plan_status(P.handle) == 2  # sticky
        P.close()
    finally:
        L.sable_debug_fail_allocations(-1)
    P = sable.plan_from(A, [(sable.VDIA, dict(a_min=50, l_seg=8)), (sable.CSR, None)], upload=False)
    assert P.info()["nnz_vdia"] > 0
    P.close()


@pytest.mark.parametrize("passes", [2, 3])
def test_multi_pass_bands_match_oracle(passes):
    """Multi-ribbon VDIA: the library's band stages per pass give exactly the
    oracle's segments, values and remainder; the far band that one pass sends
    to CSR comes back as a second-pass segment, and the plan rebuilt from its
    region table is identical."""
    A = synth.assemble(np.random.default_rng(4), 200, 260, bands=[(-1, 0, 200), (0, 0, 200), (1, 0, 200),
                                                                  (50, 0, 200)], values="int")
    ex = _compare(A, [(sable.VDIA, dict(delta=0.75, a_min=100, l_seg=16, passes=passes)), (sable.CSR, None)])
    assert sorted(ex.segments) == [(0, 200, -1, 3), (0, 200, 50, 1)]
    rng = np.random.default_rng(11)
    m = 3000
    B = synth.assemble(rng, m, m, bands=[(o, int(rng.integers(0, 800)), int(rng.integers(1500, 2200)))
                                         for o in (-2, -1, 0, 1, 2, -300, -299, 300, 301)], n_scatter=4000)
    spec = [(sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16, passes=passes)), (sable.CSR, None)]
    ex = _compare(B, spec)
    one = ox.run_plan(m, m, B["row"], B["col"], B["val"], [(ox.VDIA, ox.Params(delta=0.75, a_min=256, l_seg=16)),
                                                          (ox.CSR, None)])
    assert np.sum(ex.owner == ox.CSR) < np.sum(one.owner == ox.CSR)   # fewer entries left to CSR
    P = sable.plan_from(B, spec, upload=False)
    Q = sable.Plan(m, m, B["row"], B["col"], B["val"]).add_stages(P.region_table()).extract()
    assert np.array_equal(P.segments(), Q.segments()) and np.array_equal(P.vdia_values(), Q.vdia_values())
    assert P.region_stages()[0].max() == passes - 1
    P.close()
    Q.close()


def test_passes_rejected_outside_range_and_for_other_kinds():
    A = synth.assemble(np.random.default_rng(1), 50, 50, n_scatter=100)
    P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    for kind, passes in ((sable.VDIA, 0), (sable.VDIA, 9), (sable.VBR, 2), (sable.CSR, 2)):
        with pytest.raises(sable.SableError):
            P.add_extractor(kind, passes=passes)
    P.close()


def test_inspector_choice_rules():
    A = synth.assemble(np.random.default_rng(2), 64, 64, bands=[(0, 0, 64)], n_scatter=50)
    P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    with pytest.raises(sable.SableError) as e:
        P.set_inspector(2)
    assert e.value.status == 1
    # a block stage whose pre-pass tiles exceed what the device counts: refused, not sticky
    P.add_extractor(sable.VBR, tile=65).add_extractor(sable.CSR)
    P.set_inspector(sable.INSPECT_DEVICE)
    with pytest.raises(sable.SableError) as e:
        P.extract()
    assert e.value.status == 8
    assert P.status() == 0
    P.set_inspector(sable.INSPECT_HOST).extract()
    with pytest.raises(sable.SableError) as e:
        P.set_inspector(sable.INSPECT_DEVICE)                 # after extract
    assert e.value.status == 5
    P.close()


def test_device_inspector_without_a_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the device inspector's parity tests cover it")
    A = synth.assemble(np.random.default_rng(3), 128, 128, bands=[(0, 0, 128)], n_scatter=50)
    P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    P.add_extractor(sable.VDIA).add_extractor(sable.CSR).set_inspector(sable.INSPECT_DEVICE)
    with pytest.raises(sable.SableError) as e:
        P.extract()
    assert e.value.status == 3
    assert P.status() == 3
    P.close()
    # a plan whose stages need no device counting makes no CUDA call
    P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    P.add_extractor(sable.VBR, tile=0).add_extractor(sable.CSR).set_inspector(sable.INSPECT_DEVICE).extract()
    assert P.info()["nnz"] == A["row"].size
    P.close()


def test_release_build_refuses_the_debug_column_hook():
    """The hook that writes a column outside the matrix exists only in the
    debug build: the release library answers SABLE_ERR_UNSUPPORTED before
    looking at its arguments (no GPU needed)."""
    L = sable.lib()
    A = synth.assemble(np.random.default_rng(4), 64, 64, n_scatter=200)
    P = sable.plan_from(A, [(sable.CSR, None)], upload=False)
    assert L.sable_debug_set_csr_column(P.handle, 0, 1000) == 8
    assert L.sable_debug_set_csr_column(None, 0, 0) == 8
    P.close()


def test_debug_build_compiles_and_exports_the_same_symbols():
    """The debug build (index checks in the hot kernels) builds from the same
    sources and exports every declared entry point, like the release build."""
    import ctypes
    from paper_2407_00829_gb300 import build
    lib = build.build(checks=True)
    L = ctypes.CDLL(lib)
    hdr = open(os.path.join(ROOT, "include", "sable.h")).read()
    declared = set(re.findall(r"\b(sable_[a-z0-9_]+)\s*\(", hdr))
    assert [d for d in sorted(declared) if not hasattr(L, d)] == []
