"""FindBlock on the device (device_search = 1) chooses the same blocks as the
host search: extractions compared bit for bit on matrices whose candidate
regions are large enough for the device path."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _same(P, Q):
    assert P.info() == Q.info()
    np.testing.assert_array_equal(P.segments(), Q.segments())
    np.testing.assert_array_equal(P.blocks(), Q.blocks())
    np.testing.assert_array_equal(P.vbr_values(), Q.vbr_values())
    for a, b in zip(P.csr(), Q.csr()):
        np.testing.assert_array_equal(a, b)


def _cases():
    out = []
    for seed in range(3):
        rng = np.random.default_rng(900 + seed)
        m = 3000
        out.append(synth.assemble(rng, m, m, bands=[(o, 0, m) for o in range(-6, 6)],
                                  blocks=[(300, 1900, 180, 150, 0.85), (1200, 400, 260, 230, 0.7),
                                          (2500, 2500, 120, 400, 0.9)], n_scatter=20000))
    out.append(synth.mixed_matrix(np.random.default_rng(7), 20000, 20.0))
    return out


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("order", ["vbr_first", "vdia_first"])
def test_device_findblock_matches_host(k, order):
    A = _cases()[k]
    vbr = dict(delta=0.5, a_min=256, max_span=256)
    vd = (sable.VDIA, dict(delta=0.75, a_min=256, l_seg=16))
    for dev in (0, 1):
        spec = [(sable.VBR, dict(vbr, device_search=dev))] if order == "vbr_first" else [vd]
        spec = spec + ([vd] if order == "vbr_first" else [(sable.VBR, dict(vbr, device_search=dev))]) + [(sable.CSR, None)]
        if dev == 0:
            P = sable.plan_from(A, spec, upload=False)
        else:
            Q = sable.plan_from(A, spec, upload=False)
    assert P.info()["n_blocks"] > 0
    _same(P, Q)
    P.close()
    Q.close()


@pytest.mark.slow
def test_device_findblock_200k():
    """The 200k block workload: same 820 blocks, and the extraction time of
    both searches (printed)."""
    A = synth.blocks_scatter_200k()
    times = {}
    plans = {}
    for dev in (0, 1):
        t0 = time.perf_counter()
        plans[dev] = sable.plan_from(A, [(sable.VBR, dict(a_min=256, device_search=dev)), (sable.CSR, None)],
                                     upload=False)
        times[dev] = time.perf_counter() - t0
    print("extract seconds host / device search:", times)
    _same(plans[0], plans[1])
    assert plans[1].info()["n_blocks"] > 700
    for P in plans.values():
        P.close()
