"""GPU parity of the learned planner's device code (features, MLP forward /
backward, Adam) against the FP64 references in oracle/ml.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ml
import paper_2407_00829_gb300 as sable
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _mats():
    rng = np.random.default_rng(77)
    out = [synth.assemble(rng, 3000, 2500, bands=[(o, 0, 3000) for o in (-1, 0, 1)],
                          blocks=[(100, 200, 60, 40, 0.9)], row_lengths=synth.powerlaw_lengths(rng, 3000, kmax=300)),
           synth.mixed_matrix(rng, 5000, 40.0), synth.blocks_bands_scatter_4096()]
    return out


@pytest.mark.parametrize("k", range(3))
def test_features_match_oracle(k):
    A = _mats()[k]
    row = torch.from_numpy(A["row"]).cuda()
    col = torch.from_numpy(A["col"]).cuda()
    f = sable.features(A["m"], A["n"], row, col).cpu().numpy()
    ref = ml.features(A["m"], A["n"], A["row"], A["col"])
    np.testing.assert_allclose(f, ref, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("B", [1, 64, 300])
def test_mlp_forward_grad_adam_match_oracle(B):
    shape = (24, 32, 32, 10)
    net = sable.Mlp(*shape, seed=B)
    rng = np.random.default_rng(B)
    X = rng.standard_normal((B, 24)).astype(np.float32)
    T = rng.standard_normal((B, 10)).astype(np.float32)
    mask = (rng.random((B, 10)) < 0.6).astype(np.float32)
    p0 = net.params.cpu().numpy().astype(np.float64)
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    np.testing.assert_allclose(Y, ml.mlp_forward(shape, p0, X), rtol=1e-4, atol=1e-5)
    loss = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(mask).cuda())
    ref_loss, ref_g = ml.mlp_grad(shape, p0, X, T, mask)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    g = net.grads.cpu().numpy()
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * max(1.0, np.max(np.abs(ref_g)))
    net.adam(lr=1e-2)
    p1, _, _ = ml.adam(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, lr=1e-2)
    np.testing.assert_allclose(net.params.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)


def test_training_reduces_loss():
    shape = (24, 32, 32, 4)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((256, 24)).astype(np.float32)
    Wt = rng.standard_normal((24, 4))
    T = np.tanh(X @ Wt).astype(np.float32)
    net = sable.Mlp(*shape, seed=1)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    first = float(net.grad(Xd, Td).item())
    for _ in range(300):
        net.grad(Xd, Td)
        net.adam(lr=3e-3)
    last = float(net.grad(Xd, Td).item())
    assert last < 0.2 * first


def test_features_entry_outside_the_matrix_gives_nan_and_no_stray_write():
    # one column index past n and one negative row: the kernels skip both
    # (bounds-checked) and every feature comes back NaN; a valid call
    # afterwards is exact again
    A = _mats()[1]
    row = A["row"].copy()
    col = A["col"].copy()
    col[5] = A["n"] + 3
    row[9] = -1
    f = sable.features(A["m"], A["n"], torch.from_numpy(row).cuda(), torch.from_numpy(col).cuda()).cpu().numpy()
    assert np.isnan(f).all()
    good = sable.features(A["m"], A["n"], torch.from_numpy(A["row"]).cuda(),
                          torch.from_numpy(A["col"]).cuda()).cpu().numpy()
    np.testing.assert_allclose(good, ml.features(A["m"], A["n"], A["row"], A["col"]), rtol=1e-5, atol=1e-6)
