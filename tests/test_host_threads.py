"""The host extraction's threaded paths (COO ingest, residual and transposed
residual, the block pre-pass's cell counts, FindBlock's outer loop, FitRibbon)
give exactly the single-threaded plan: the same matrix extracted in two child
processes, SABLE_THREADS=1 and SABLE_THREADS=4, on a matrix large enough
(> 2^20 entries, duplicates included) for every threaded path to run."""
import os
import subprocess
import sys

import numpy as np

from conftest import ROOT

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_2407_00829_gb300 as sable
import synth
rng = np.random.default_rng(17)
m = 60000
A = synth.assemble(rng, m, m, bands=[(0, 0, m), (1, 100, m - 200), (-1, 0, m), (7, 5000, 30000)],
                   blocks=[(1000, 3000, 120, 150, 0.8), (20000, 41000, 200, 90, 0.9), (45000, 2000, 64, 64, 1.0)],
                   n_scatter=1200000)
# duplicates in the input: the first 50000 entries again, in reverse order
row = np.concatenate([A["row"], A["row"][:50000][::-1]])
col = np.concatenate([A["col"], A["col"][:50000][::-1]])
val = np.concatenate([A["val"], rng.uniform(-1, 1, 50000).astype(np.float32)])
assert row.size > (1 << 20)
P = sable.Plan(m, m, row, col, val)
P.add_extractor(sable.VDIA, delta=0.6, a_min=256).add_extractor(sable.VBR, a_min=400, coverage_min=0.0).add_extractor(sable.CSR)
P.extract()
rp, ci, cv = P.csr()
np.savez({out!r}, segs=P.segments(), blks=P.blocks(), vd=P.vdia_values(), vb=P.vbr_values(), rp=rp, ci=ci, cv=cv)
"""


def _run(threads, out):
    env = dict(os.environ, SABLE_THREADS=str(threads))
    code = CHILD.format(root=ROOT, out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_threaded_extraction_equals_single_threaded(tmp_path):
    one = _run(1, str(tmp_path / "t1.npz"))
    four = _run(4, str(tmp_path / "t4.npz"))
    for k in ("segs", "blks", "vd", "vb", "rp", "ci", "cv"):
        assert np.array_equal(one[k], four[k]), k
    assert one["segs"].shape[0] > 0 and one["blks"].shape[0] >= 2
