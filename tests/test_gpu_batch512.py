"""The batched workload's generator (rows log-uniform in [1k, 64k], 5-200
entries per row, mixed band / block / scatter): a sample of its matrices in
one grouped launch, every output row checked against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2407_00829_gb300 as sable
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_batch512_sample():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    mats = synth.batch_512(count=24)
    plans = [sable.plan_from(A, [(sable.VDIA, None), (sable.VBR, dict(a_min=256)), (sable.CSR, None)])
             for A in mats]
    B = sable.Batch(plans)
    xs = [torch.from_numpy(synth.dense_operand(i, A["n"])).cuda() for i, A in enumerate(mats)]
    ys = [torch.empty(A["m"], device="cuda") for A in mats]
    g = B.graph_spmv(xs, ys)
    g.launch()
    Bs = [torch.from_numpy(synth.dense_operand(50 + i, A["n"], 32)).cuda() for i, A in enumerate(mats)]
    Cs = [torch.empty(A["m"], 32, device="cuda") for A in mats]
    B.spmm(Bs, Cs, 32, sable.BF16_BLOCKS)
    torch.cuda.synchronize()
    for A, x, y, b, c in zip(mats, xs, ys, Bs, Cs):
        ref = oracle.spmv(A["m"], A["row"], A["col"], A["val"], x.cpu().numpy())
        assert oracle.normwise_err(y.cpu().numpy(), ref) <= 1e-5
        refC = oracle.spmm(A["m"], A["row"], A["col"], A["val"], b.cpu().numpy())
        assert oracle.normwise_err(c.cpu().numpy(), refC) <= 2e-2
    assert B.device_error() == 0
    g.close()
    B.close()
    for P in plans:
        P.close()
