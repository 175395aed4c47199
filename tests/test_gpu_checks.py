"""The debug build (SABLE_CHECKS): its kernels test every gathered column
against the matrix's width.  On valid plans it computes what the release
build does and records nothing; with one CSR remainder column overwritten to
lie outside the matrix (the debug hook, refused by the release build) the
SpMV and the row-split SpMM record SABLE_ERR_KERNEL with the check's tag,
the index and its bound, skip that entry, and compute the rest correctly.
The checks run in a child process that loads the debug build."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import torch
import paper_2407_00829_gb300 as sable
import oracle, synth
torch.cuda.set_device(0)
A = synth.blocks_bands_scatter_4096()
m, n = A["m"], A["n"]
spec = [(sable.VDIA, None), (sable.VBR, None), (sable.CSR, None)]
x_np = synth.dense_operand(11, n)
B_np = synth.dense_operand(12, n, 64)
ref = oracle.spmv(m, A["row"], A["col"], A["val"], x_np)
refm = oracle.spmm(m, A["row"], A["col"], A["val"], B_np)
x = torch.from_numpy(x_np).cuda()
B = torch.from_numpy(B_np).cuda()
out = {{}}

def run(P, what):
    if what == "spmv":
        y = torch.empty(m, device="cuda")
        P.spmv(x, y)
    else:
        y = torch.empty(m, 64, device="cuda")
        P.spmm(B, y, sable.FP32)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)

P = sable.plan_from(A, spec)
out["clean"] = {{"spmv_err": oracle.normwise_err(run(P, "spmv"), ref),
                 "spmm_err": oracle.normwise_err(run(P, "spmm"), refm), "word": P.device_error()}}
rp, ci, cv = P.csr()
e = int(rp[m // 2])                       # the first remainder entry of a middle row (or the next)
r = int(np.searchsorted(rp, e, side="right") - 1)
col, val = int(ci[e]), float(cv[e])
P.close()
for what in ("spmv", "spmm"):
    P = sable.plan_from(A, spec)
    P.debug_set_csr_column(e, n + 7)
    y = run(P, what)
    exp = (ref.copy() if what == "spmv" else refm.copy())
    exp[r] -= val * (x_np[col] if what == "spmv" else B_np[col].astype(np.float64))
    out[what] = {{"word": P.device_error(), "err_without_entry": oracle.normwise_err(y, exp)}}
    P.close()
out["n"] = n
print(json.dumps(out))
"""


def test_debug_build_checks_columns_and_records_the_bad_one():
    from paper_2407_00829_gb300 import build
    lib = build.build(checks=True)
    env = dict(os.environ, SABLE_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    n = d["n"]
    assert d["clean"]["word"] == [0, 0, 0, 0]
    assert d["clean"]["spmv_err"] <= 1e-5 and d["clean"]["spmm_err"] <= 1e-5
    assert d["spmv"]["word"] == [7, 1, n + 7, n]          # SABLE_ERR_KERNEL, SpMV CSR column
    assert d["spmm"]["word"] == [7, 3, n + 7, n]          # SABLE_ERR_KERNEL, SpMM CSR column
    assert d["spmv"]["err_without_entry"] <= 1e-5
    assert d["spmm"]["err_without_entry"] <= 1e-5


def test_release_build_refuses_the_debug_hook():
    import torch
    import paper_2407_00829_gb300 as sable
    import synth
    A = synth.blocks_bands_scatter_4096()
    P = sable.plan_from(A, [(sable.VDIA, None), (sable.CSR, None)])
    with pytest.raises(sable.SableError) as e:
        P.debug_set_csr_column(0, A["n"] + 7)
    assert e.value.status == 8
    assert P.device_error() == [0, 0, 0, 0]
    P.close()
