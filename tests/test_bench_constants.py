"""The bench's committed per-workload byte counts (used by its reference arm,
which loads no part of the library) equal the algorithmic bytes of the
library's plans of those seeded workloads, extracted here on the host."""
import os
import sys

import pytest

import paper_2407_00829_gb300 as sable
import synth
from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("workload", ["spmv4096", "spmv1m"])
def test_workload_bytes_constant(workload):
    A, ex, _desc, _x = bench._workload(workload)
    kinds = [sable.VDIA, sable.VBR, sable.CSR] if ex == "VDIA+VBR+CSR" else [sable.VDIA, sable.CSR]
    P = sable.plan_from(A, [(k, None) for k in kinds], upload=False)
    assert P.info()["spmv_bytes"] == bench.WORKLOAD_BYTES[workload]
    P.close()


def test_reference_arm_imports_no_library_code():
    src = open(os.path.join(ROOT, "bench.py")).read()
    body = src[src.index("def run_reference("):]
    body = body[:body.index("\ndef ", 1)]
    assert "paper_2407_00829_gb300" not in body and "sable." not in body
