"""sable_features_noalloc: the feature kernels run on a fixed device array
instead of a caller workspace, for callers that may not allocate device memory
(a host framework owning all GPU memory through its own pool, a plugin that
only receives input and output pointers, latency-critical code that cannot
take the synchronisation cudaMalloc may cause).

The GPU test calls it through the C ABI twice in a row, on a larger matrix and
then on a smaller one (so stale counters from the first call would show up in
the second), and compares each result with sable_features, which takes a
caller workspace.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_00829_gb300 as sable
import synth

MAX_BYTES = 32 << 20


def _noalloc():
    f = sable.lib().sable_features_noalloc
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [i64, i64, i64, p, p, p, p]
    f.restype = ctypes.c_int32
    return f


def test_rejects_sizes_beyond_the_fixed_array():
    L = sable.lib()
    assert L.sable_features_workspace_bytes(700_000, 700_000, 1 << 20) > MAX_BYTES
    # rejected on the host before any device work: the pointers are never used
    h = np.zeros(64, np.int32)
    a = h.ctypes.data
    assert _noalloc()(700_000, 700_000, 1 << 20, a, a, a, None) == 8          # SABLE_ERR_UNSUPPORTED
    assert _noalloc()(10, 10, (1 << 20) + 1, a, a, a, None) == 8
    assert _noalloc()(-1, 10, 0, None, None, a, None) == 1                    # SABLE_ERR_INVALID
    assert _noalloc()(10, 10, 0, None, None, None, None) == 1


@pytest.mark.gpu
def test_noalloc_matches_workspace_features_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    rng = np.random.default_rng(2024)
    mats = [synth.assemble(rng, 40_000, 36_000, bands=[(o, 0, 36_000) for o in (-2, 0, 3)],
                           blocks=[(1000, 2000, 200, 150, 0.9), (20_000, 5000, 96, 320, 0.7)],
                           row_lengths=synth.powerlaw_lengths(rng, 40_000, kmax=400)),
            synth.mixed_matrix(rng, 6000, 30.0)]
    f = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    for A in mats:
        assert sable.lib().sable_features_workspace_bytes(A["m"], A["n"], A["row"].size) <= MAX_BYTES
        row = torch.from_numpy(np.ascontiguousarray(A["row"], dtype=np.int32)).cuda()
        col = torch.from_numpy(np.ascontiguousarray(A["col"], dtype=np.int32)).cuda()
        out = torch.full((sable.NFEAT,), float("nan"), device="cuda")
        st = f(A["m"], A["n"], A["row"].size, row.data_ptr(), col.data_ptr(), out.data_ptr(), stream)
        assert st == 0, sable.STATUS.get(st, st)
        got = out.cpu().numpy()
        ref = sable.features(A["m"], A["n"], row, col).cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)


@pytest.mark.gpu
def test_noalloc_entry_outside_the_matrix_then_a_valid_call():
    # an index outside the matrix is skipped by the kernels' own check (never
    # used to address the shared array) and turns every feature into NaN;
    # the next valid call on the same array is exact again
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    A = synth.mixed_matrix(np.random.default_rng(9), 5000, 20.0)
    f = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    row = np.ascontiguousarray(A["row"], dtype=np.int32)
    col = np.ascontiguousarray(A["col"], dtype=np.int32)
    bad = col.copy()
    bad[3] = A["n"]
    for c, expect_nan in ((bad, True), (col, False)):
        rd, cd = torch.from_numpy(row).cuda(), torch.from_numpy(c).cuda()
        out = torch.zeros(sable.NFEAT, device="cuda")
        assert f(A["m"], A["n"], row.size, rd.data_ptr(), cd.data_ptr(), out.data_ptr(), stream) == 0
        got = out.cpu().numpy()
        if expect_nan:
            assert np.isnan(got).all()
        else:
            ref = sable.features(A["m"], A["n"], rd, cd).cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
