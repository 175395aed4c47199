import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload")


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: '#' comments, 'key: v v v' lines and
    a 'matrix:' block of whitespace-separated rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, mat, in_mat = {}, [], False
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line == "matrix:":
                in_mat = True
                continue
            if ":" in line:
                in_mat = False
                k, v = line.split(":", 1)
                out[k.strip()] = [float(t) for t in v.split()]
                continue
            if in_mat:
                mat.append([float(t) for t in line.split()])
    out["matrix"] = mat
    return out
