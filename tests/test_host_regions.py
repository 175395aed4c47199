"""Region tables: a plan rebuilt from the saved regions of an extraction
(sable_plan_add_regions, sable_plan_get_region_stages) equals the extraction
exactly; sable_plan_reset starts a plan over from its matrix; invalid region
stages are rejected.  Host only."""
import numpy as np
import pytest

import paper_2407_00829_gb300 as sable
import synth

V, B, C = sable.VDIA, sable.VBR, sable.CSR


def _same(P, Q):
    assert P.info() == Q.info()
    np.testing.assert_array_equal(P.segments(), Q.segments())
    np.testing.assert_array_equal(P.blocks(), Q.blocks())
    np.testing.assert_array_equal(P.vdia_values(), Q.vdia_values())
    np.testing.assert_array_equal(P.vbr_values(), Q.vbr_values())
    for a, b in zip(P.csr(), Q.csr()):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(P.region_stages(), Q.region_stages()):
        np.testing.assert_array_equal(a, b)


def _matrix(seed, m=600):
    rng = np.random.default_rng(seed)
    return synth.assemble(rng, m, m, bands=[(o, 0, m) for o in (-3, -2, -1, 0, 1, 2, 3)] + [(90, 50, 400)],
                          blocks=[(100, 300, 40, 48, 0.9), (400, 20, 64, 30, 0.85)], n_scatter=900)


PLANS = [
    [(V, dict(delta=0.75, a_min=200, l_seg=16)), (B, dict(delta=0.5, a_min=200, max_span=64)), (C, None)],
    [(B, dict(delta=0.5, a_min=200, max_span=64)), (V, dict(delta=0.75, a_min=200, l_seg=16)), (C, None)],
    [(V, dict(delta=0.6, a_min=100, l_seg=8)), (V, dict(delta=0.9, a_min=100, l_seg=8)), (C, None)],
]


@pytest.mark.parametrize("k", range(len(PLANS)))
def test_rebuild_from_region_table_is_exact(k, tmp_path):
    A = _matrix(11 + k)
    P = sable.plan_from(A, PLANS[k], upload=False)
    table = P.region_table()
    assert sum(len(g) for _, g in table) == P.info()["n_segments"] + P.info()["n_blocks"] > 0
    path = tmp_path / "t.npz"
    sable.save_region_table(path, table, A["m"], A["n"], A["row"].size)
    table2, shape = sable.load_region_table(path)
    assert shape == (A["m"], A["n"], A["row"].size)
    Q = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"]).add_stages(table2).extract()
    _same(P, Q)
    # new values, same structure: the saved regions still partition the entries
    A2 = dict(A, val=np.random.default_rng(5).standard_normal(A["row"].size).astype(np.float32))
    P2 = sable.plan_from(A2, PLANS[k], upload=False)
    Q2 = sable.Plan(A2["m"], A2["n"], A2["row"], A2["col"], A2["val"]).add_stages(table).extract()
    _same(P2, Q2)
    for X in (P, Q, P2, Q2):
        X.close()


def test_reset_gives_a_fresh_plan():
    A = _matrix(3)
    P = sable.plan_from(A, PLANS[0], upload=False)
    P.reset()
    with pytest.raises(sable.SableError):
        P.info()                                        # not extracted any more
    for kind, kw in PLANS[1]:
        P.add_extractor(kind, **(kw or {}))
    P.extract()
    Q = sable.plan_from(A, PLANS[1], upload=False)
    _same(P, Q)
    P.close()
    Q.close()


def test_overlapping_given_regions_first_claims():
    m = 64
    r, c = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    A = dict(m=m, n=m, row=r.ravel().astype(np.int32), col=c.ravel().astype(np.int32),
             val=np.arange(1, m * m + 1, dtype=np.float32))
    P = sable.Plan(m, m, A["row"], A["col"], A["val"])
    P.add_regions(B, [[0, 32, 0, 32], [16, 32, 16, 32]]).add_extractor(C).extract()
    info = P.info()
    assert info["nnz_vbr"] == 32 * 32 + 32 * 32 - 16 * 16 and info["vbr_cells"] == 2 * 32 * 32
    second = P.vbr_values()[32 * 32:].reshape(32, 32).T      # column-major block (rows 16..47, cols 16..47)
    assert np.all(second[:16, :16] == 0)                       # overlap went to the first block
    assert second[16, 16] == A["val"][(32 * m) + 32]
    P.close()


def test_invalid_region_stages():
    A = synth.assemble(np.random.default_rng(1), 100, 100, bands=[(0, 0, 100)], n_scatter=300)
    P = sable.Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    bad = [(V, [[0, 0, 0, 1]]), (V, [[90, 20, 0, 1]]), (V, [[0, 10, -100, 1]]), (V, [[0, 10, 99, 2]]),
           (B, [[0, 10, 95, 6]]), (B, [[-1, 10, 0, 6]]), (B, [[0, 10, 0, 0]]), (C, [[0, 1, 0, 1]])]
    for kind, g in bad:
        with pytest.raises(sable.SableError) as e:
            P.add_regions(kind, g)
        assert e.value.status == 1
    P.add_regions(V, [[0, 100, -99, 199]]).add_extractor(C).extract()    # every offset: all in VDIA
    assert P.info()["nnz_vdia"] == P.info()["nnz"]
    with pytest.raises(sable.SableError) as e:
        P.add_regions(B, [[0, 1, 0, 1]])
    assert e.value.status == 5
    P.close()


@pytest.mark.parametrize("k", range(len(PLANS)))
def test_update_values_equals_a_fresh_plan(k):
    A = _matrix(40 + k)
    # duplicates: repeat a tenth of the entries (summed at creation and at update)
    rng = np.random.default_rng(k)
    dup = rng.choice(A["row"].size, A["row"].size // 10, replace=False)
    A = dict(A, row=np.concatenate([A["row"], A["row"][dup]]), col=np.concatenate([A["col"], A["col"][dup]]),
             val=np.concatenate([A["val"], A["val"][dup]]))
    P = sable.plan_from(A, PLANS[k], upload=False)
    v2 = rng.standard_normal(A["row"].size).astype(np.float32)
    P.update_values(v2)
    Q = sable.plan_from(dict(A, val=v2), PLANS[k], upload=False)
    _same(P, Q)
    P.close()
    Q.close()
