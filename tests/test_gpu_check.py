"""The FP64 device reduction of the accuracy check against numpy in FP64."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_00829_gb300 as sable


def test_error_norms_rejects_bad_arguments():
    L = sable.lib()
    wb = L.sable_error_workspace_bytes()
    assert wb > 0
    h = np.zeros(8)
    a = h.ctypes.data
    assert L.sable_error_norms(None, None, 10, a, a, wb, None) == 1       # y, ref missing
    assert L.sable_error_norms(a, a, -1, a, a, wb, None) == 1
    assert L.sable_error_norms(a, a, 10, a, a, wb - 1, None) == 1          # workspace too small
    assert L.sable_error_norms(a, a, 10, None, a, wb, None) == 1


@pytest.mark.gpu
@pytest.mark.parametrize("count", [0, 1, 1000, 1_000_003])
def test_error_norms_match_numpy(count):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(count + 1)
    ref = rng.standard_normal(count) * 10.0 ** rng.uniform(-3, 3, count)
    y = (ref * (1 + 1e-6 * rng.standard_normal(count))).astype(np.float32)
    r = sable.error_norms(torch.from_numpy(y).cuda(), torch.from_numpy(ref).cuda())
    e = y.astype(np.float64) - ref
    if count == 0:
        assert r["max_abs_err"] == r["max_abs_ref"] == r["sq_err"] == r["sq_ref"] == 0.0
        return
    assert r["max_abs_err"] == np.max(np.abs(e))
    assert r["max_abs_ref"] == np.max(np.abs(ref))
    assert r["sq_err"] == pytest.approx(np.sum(e * e), rel=1e-12)
    assert r["sq_ref"] == pytest.approx(np.sum(ref * ref), rel=1e-12)
    r2 = sable.error_norms(torch.from_numpy(y).cuda(), torch.from_numpy(ref).cuda())
    assert r2 == r                                                          # fixed-order reduction


@pytest.mark.gpu
def test_error_norms_nan_shows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    y = torch.ones(5000, device="cuda")
    y[3777] = float("nan")
    r = sable.error_norms(y, torch.ones(5000, dtype=torch.float64, device="cuda"))
    assert np.isnan(r["max_abs_err"]) and np.isnan(r["normwise"])
