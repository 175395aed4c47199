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
