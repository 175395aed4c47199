"""FP64 CPU oracle for the hybrid VDIA+VBR+CSR SpMV/SpMM path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_2407_00829_gb300``) and neither
package imports the other.

Contents
--------
* ``spmv`` / ``spmm`` / ``spmm_rows`` -- the plain definitions of the two
  kernels evaluated in Section 5 ("Kernels"): y_i = sum_j A_ij x_j and
  C = A B, computed in FP64 straight from the COO triples (``sable_oracle.c``).
* ``normwise_err`` -- the accuracy measure ||y - y_ref||_inf / ||y_ref||_inf.
* ``bf16_round`` -- round-to-nearest-even to bfloat16, written from the
  definition of the format (8 exponent bits, 7 stored mantissa bits).
* ``formats`` -- the VDIA (Section 4.2.1, Fig. 4) and VBR (Appendix B,
  Fig. 9) layouts built from a given partition.
* ``extract`` -- the extractors: CSR (Appendix A.1), the band extractor
  (Algorithms 3 and 4 with a FitRibbon reading) and the block partitioner
  (Algorithms 1 and 2), plus the exact partition checker.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sable_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def build() -> str:
    """Compile the C oracle with gcc (plain -O2, no vector or fast-math flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def build_omp():
    """The same C file with -fopenmp (the all-cores CPU baseline); None when
    the host compiler has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not os.path.exists(_SO_OMP)) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC):
        tmp = _SO_OMP + f".{os.getpid()}.tmp"
        r = subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                            "-fopenmp", _SRC, "-o", tmp], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def _bind(lib):
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.oracle_spmv_coo.argtypes = [i64, i64, p, p, p, p, p]
    lib.oracle_spmv_coo_f32.argtypes = [i64, i64, p, p, p, p, p]
    lib.oracle_spmm_coo_f32.argtypes = [i64, i64, p, p, p, p, i64, i64, p, i64]
    lib.oracle_spmm_coo_rows_f32.argtypes = [i64, i64, p, p, p, p, i64, i64, i64, p, p, p]
    lib.oracle_coo_rows.argtypes = [i64, i64, p, p, p]
    lib.oracle_spmv_rows_f32.argtypes = [i64, p, p, p, p, p, p]
    for f in (lib.oracle_spmv_coo, lib.oracle_spmv_coo_f32, lib.oracle_spmm_coo_f32,
              lib.oracle_spmm_coo_rows_f32, lib.oracle_coo_rows, lib.oracle_spmv_rows_f32):
        f.restype = None
    lib.oracle_threads.argtypes = []
    lib.oracle_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            so = build_omp()
            _lib_omp = _bind(ctypes.CDLL(so)) if so else False
    return _lib_omp or None


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _coo(row, col, val, dtype):
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=dtype)
    if not (row.shape == col.shape == val.shape):
        raise ValueError("COO arrays differ in length")
    return row, col, val


def spmv(m: int, row, col, val, x) -> np.ndarray:
    """y = A x in FP64 from COO triples (duplicates add up).

    FP32 ``val``/``x`` are widened exactly per term; FP64 inputs are used as is.
    """
    lib = _load()
    y = np.empty(int(m), dtype=np.float64)
    if np.asarray(val).dtype == np.float64 or np.asarray(x).dtype == np.float64:
        row, col, val = _coo(row, col, val, np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        lib.oracle_spmv_coo(int(m), val.size, _ptr(row), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    else:
        row, col, val = _coo(row, col, val, np.float32)
        x = np.ascontiguousarray(x, dtype=np.float32)
        lib.oracle_spmv_coo_f32(int(m), val.size, _ptr(row), _ptr(col), _ptr(val), _ptr(x),
                                _ptr(y))
    return y


class RowOrder:
    """The COO triples grouped by row (stable counting sort, input order kept
    within a row), for the row-loop form of y = A x."""

    def __init__(self, m: int, row, col, val):
        self.m = int(m)
        self.row, self.col, self.val = _coo(row, col, val, np.float32)
        self.rp = np.empty(self.m + 1, dtype=np.int64)
        self.perm = np.empty(self.row.size, dtype=np.int64)
        _load().oracle_coo_rows(self.m, self.row.size, _ptr(self.row), self.rp.ctypes.data,
                                self.perm.ctypes.data)

    def spmv(self, x, threads: bool = False) -> np.ndarray:
        """y = A x in FP64, one row at a time: identical to ``spmv`` (same
        terms in the same order per row).  threads=True runs the OpenMP build
        over the rows on every host core; raises if there is none."""
        lib = _load_omp() if threads else _load()
        if lib is None:
            raise RuntimeError("the C oracle could not be built with OpenMP")
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.empty(self.m, dtype=np.float64)
        lib.oracle_spmv_rows_f32(self.m, self.rp.ctypes.data, self.perm.ctypes.data, _ptr(self.col),
                                 _ptr(self.val), _ptr(x), _ptr(y))
        return y


def omp_threads() -> int:
    """Threads the OpenMP build of the oracle runs (0 if it could not be built)."""
    lib = _load_omp()
    return int(lib.oracle_threads()) if lib else 0


def spmm(m: int, row, col, val, B) -> np.ndarray:
    """C = A B in FP64; B is a dense row-major FP32 matrix (n x N)."""
    lib = _load()
    row, col, val = _coo(row, col, val, np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    N = B.shape[1]
    C = np.empty((int(m), N), dtype=np.float64)
    lib.oracle_spmm_coo_f32(int(m), val.size, _ptr(row), _ptr(col), _ptr(val), _ptr(B), N, N,
                            _ptr(C), N)
    return C


def spmm_rows(m: int, row, col, val, B, sel) -> np.ndarray:
    """Rows ``sel`` of C = A B in FP64 (for sampled checks of huge products)."""
    lib = _load()
    row, col, val = _coo(row, col, val, np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    sel = np.asarray(sel, dtype=np.int64)
    uniq, back = np.unique(sel, return_inverse=True)   # the C routine wants distinct rows
    uniq = np.ascontiguousarray(uniq)
    N = B.shape[1]
    slot = np.empty(int(m), dtype=np.int64)
    out = np.empty((uniq.size, N), dtype=np.float64)
    lib.oracle_spmm_coo_rows_f32(int(m), val.size, _ptr(row), _ptr(col), _ptr(val), _ptr(B),
                                 N, N, uniq.size, _ptr(uniq), _ptr(slot), _ptr(out))
    return out[back]


def normwise_err(y, y_ref) -> float:
    """||y - y_ref||_inf / ||y_ref||_inf over every element (0 if both vanish)."""
    y = np.asarray(y, dtype=np.float64).ravel()
    y_ref = np.asarray(y_ref, dtype=np.float64).ravel()
    den = float(np.max(np.abs(y_ref))) if y_ref.size else 0.0
    num = float(np.max(np.abs(y - y_ref))) if y_ref.size else 0.0
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as FP32.

    bfloat16 keeps the top 16 bits of the IEEE-754 binary32 pattern.  Adding
    0x7FFF plus the lowest kept bit to the pattern and truncating implements
    round-to-nearest with ties to the even kept pattern; NaN stays NaN.
    """
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = a[nan]
    return out


def pow2_scale(amax: float) -> float:
    """Per-block power-of-two scale s = 2^ceil(log2 amax) (1 for an all-zero block)."""
    if not (amax > 0.0):
        return 1.0
    m, e = np.frexp(np.float64(amax))  # amax = m * 2^e, m in [0.5, 1)
    return float(np.ldexp(1.0, int(e) - 1)) if m == 0.5 else float(np.ldexp(1.0, int(e)))


from . import formats, extract  # noqa: E402,F401
