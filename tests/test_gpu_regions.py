"""A plan rebuilt from a saved region table computes what the extracted plan
computes on the device; a reset plan can be extracted and uploaded again.
(The host tables of the two plans are compared bit for bit on the CPU; on the
device the VBR part sums warp partials with shared-memory atomics, whose
order varies from run to run, so the results agree to FP32 rounding.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth
from test_host_regions import PLANS, _matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _run(P, x, B):
    y = torch.full((P.m,), float("nan"), device="cuda")
    C = torch.full((P.m, B.shape[1]), float("nan"), device="cuda")
    P.spmv(x, y)
    P.spmm(B, C, sable.FP32)
    torch.cuda.synchronize()
    return y.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("k", range(len(PLANS)))
def test_rebuilt_plan_matches(k):
    A = _matrix(21 + k)
    P = sable.plan_from(A, PLANS[k])
    Q = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"]).add_stages(P.region_table()).extract().upload()
    xs = synth.dense_operand(3, A["n"])
    Bs = synth.dense_operand(4, A["n"], 24)
    x, B = torch.from_numpy(xs).cuda(), torch.from_numpy(Bs).cuda()
    yp, cp = _run(P, x, B)
    yq, cq = _run(Q, x, B)
    assert oracle.normwise_err(yq, yp) <= 1e-6
    assert oracle.normwise_err(cq, cp) <= 1e-6
    assert oracle.normwise_err(yq, oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs)) <= 1e-5
    # the same plan object, reset and extracted with another plan
    Q.reset()
    Q.add_stages(sable.plan_from(A, PLANS[(k + 1) % len(PLANS)], upload=False).region_table()).extract().upload()
    yr, cr = _run(Q, x, B)
    assert oracle.normwise_err(yr, oracle.spmv(A["m"], A["row"], A["col"], A["val"], xs)) <= 1e-5
    assert oracle.normwise_err(cr, oracle.spmm(A["m"], A["row"], A["col"], A["val"], Bs)) <= 1e-5
    P.close()
    Q.close()


@pytest.mark.parametrize("k", range(len(PLANS)))
def test_update_values_on_the_device(k):
    A = _matrix(31 + k)
    P = sable.plan_from(A, PLANS[k])
    v2 = np.random.default_rng(k).uniform(-2, 2, A["row"].size).astype(np.float32)
    P.update_values(v2)
    xs = synth.dense_operand(5, A["n"])
    Bs = synth.dense_operand(6, A["n"], 64)
    y, C = _run(P, torch.from_numpy(xs).cuda(), torch.from_numpy(Bs).cuda())
    assert oracle.normwise_err(y, oracle.spmv(A["m"], A["row"], A["col"], v2, xs)) <= 1e-5
    refC = oracle.spmm(A["m"], A["row"], A["col"], v2, Bs)
    assert oracle.normwise_err(C, refC) <= 1e-5
    Cb = torch.empty(A["m"], 64, device="cuda")
    P.spmm(torch.from_numpy(Bs).cuda(), Cb, sable.BF16_BLOCKS)
    torch.cuda.synchronize()
    assert oracle.normwise_err(Cb.cpu().numpy(), refC) <= 2e-2
    yp = torch.empty(A["m"], device="cuda")
    P.csr_spmv(torch.from_numpy(xs).cuda(), yp)
    torch.cuda.synchronize()
    assert oracle.normwise_err(yp.cpu().numpy(), oracle.spmv(A["m"], A["row"], A["col"], v2, xs)) <= 1e-5
    P.close()


def test_injected_device_allocation_failures_return_oom():
    """The upload's host staging and device allocation, and a batch's device
    allocation, fail on request with SABLE_ERR_OOM; nothing is left
    half-built and later uploads and batches work."""
    import numpy as np
    import synth
    L = sable.lib()
    A = synth.mixed_matrix(np.random.default_rng(8), 1500, 12.0)
    spec = [(sable.VDIA, None), (sable.CSR, None)]
    try:
        for after in (0, 1):                       # 0: host staging, 1: device allocation
            P = sable.plan_from(A, spec, upload=False)
            L.sable_debug_fail_allocations(after)
            assert L.sable_plan_upload(P.handle, None) == 2
            L.sable_debug_fail_allocations(-1)
            P.close()
        P = sable.plan_from(A, spec)
        L.sable_debug_fail_allocations(0)
        import ctypes
        arr = (ctypes.c_void_p * 1)(P.handle)
        h = ctypes.c_void_p()
        assert L.sable_batch_create(arr, 1, ctypes.byref(h)) == 2 and not h.value
    finally:
        L.sable_debug_fail_allocations(-1)
    B = sable.Batch([P])
    x = torch.from_numpy(synth.dense_operand(1, A["n"])).cuda()
    y = torch.empty(A["m"], device="cuda")
    B.spmv([x], [y])
    torch.cuda.synchronize()
    ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x.cpu().numpy())
    assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
    B.close()
    P.close()
