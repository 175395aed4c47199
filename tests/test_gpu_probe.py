"""Calibration kernels: the random-gather probes run, and the row probe
rejects shapes it does not handle (host-side checks, nothing launched)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2407_00829_gb300 as sable

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_gather_probes_run():
    x = torch.rand(100_003, device="cuda")
    out = torch.zeros(1, device="cuda")
    sable.probe_gather(x, 1 << 20, out)
    for n, N in ((5000, 128), (777, 36), (64, 4)):
        B = torch.rand(n, N, device="cuda")
        sable.probe_row_gather(B, 100_000, out)
        sable.probe_row_gather(B, 0, out)
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape", [(100, 130), (100, 2), (100, 6)])
def test_row_probe_rejects(shape):
    B = torch.rand(*shape, device="cuda")
    out = torch.zeros(1, device="cuda")
    with pytest.raises(sable.SableError):
        sable.probe_row_gather(B, 1000, out)


def test_bulk_copy_gather_probe_runs():
    x = torch.rand(1_000_003, device="cuda")
    out = torch.zeros(1, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for count in (0, 1, 255, 257, 1 << 20):
        sable.probe_bulk_gather(x, count, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """A wait that nothing satisfies ends with SABLE_ERR_TIMEOUT at the set
    budget (no copy or tensor-core work in flight); afterwards the device
    still runs the library's kernels."""
    import numpy as np
    import oracle
    import synth
    old = sable.wait_limit()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        sable.set_wait_limit(2_000_000)              # ~1 ms
        sable.probe_wait_limit(status)
        torch.cuda.synchronize()
        assert int(status.item()) == 6               # SABLE_ERR_TIMEOUT
    finally:
        sable.set_wait_limit(old)
    assert sable.wait_limit() == old
    A = synth.mixed_matrix(np.random.default_rng(3), 2000, 10.0)
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.CSR, None)])
    x = synth.dense_operand(1, A["n"])
    y = torch.empty(A["m"], device="cuda")
    P.spmv(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert oracle.normwise_err(y.cpu().numpy(), oracle.spmv(A["m"], A["row"], A["col"], A["val"], x)) <= 1e-5
    P.close()
