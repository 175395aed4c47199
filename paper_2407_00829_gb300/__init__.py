"""Python binding of libsable (include/sable.h): argument marshalling only.

Every SpMV/SpMM step runs in the library's CUDA kernels; PyTorch supplies
device memory and streams.  Loading fails loudly when the library is missing
(there is no CPU fallback): build it with ``paper_2407_00829_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library this process loads: the release build, or another build (the
# debug build, _build_checks/libsable.so) named by SABLE_LIB_PATH
LIB_PATH = os.environ.get("SABLE_LIB_PATH") or os.path.join(_HERE, "_build", "libsable.so")

VDIA, VBR, CSR = 0, 1, 2
FP32, BF16_BLOCKS, FP32_SPLIT = 0, 1, 2
INSPECT_HOST, INSPECT_DEVICE = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA runtime error",
          4: "incomplete plan", 5: "call out of order", 6: "device wait timed out",
          7: "kernel bounds check failed", 8: "unsupported"}

EXPORTED = [
    "sable_default_params", "sable_plan_create", "sable_plan_add_extractor", "sable_extract",
    "sable_plan_upload", "sable_spmv", "sable_spmm", "sable_csr_spmv", "sable_csr_spmm",
    "sable_plan_info", "sable_plan_get_segments", "sable_plan_get_blocks",
    "sable_plan_get_vdia_values", "sable_plan_get_vbr_values", "sable_plan_get_csr",
    "sable_plan_set_tiling", "sable_plan_status", "sable_plan_destroy", "sable_status_string",
    "sable_probe_gather", "sable_probe_row_gather", "sable_batch_create", "sable_batch_spmv", "sable_batch_spmm",
    "sable_batch_graph_spmv", "sable_batch_graph_spmm", "sable_graph_launch", "sable_graph_destroy",
    "sable_batch_status", "sable_batch_destroy", "sable_features_workspace_bytes", "sable_features",
    "sable_mlp_param_count", "sable_mlp_work_floats", "sable_mlp_forward", "sable_mlp_grad", "sable_mlp_adam",
    "sable_plan_add_regions", "sable_plan_get_region_stages", "sable_plan_reset",
    "sable_error_workspace_bytes", "sable_error_norms", "sable_plan_get_tiling", "sable_autotune",
    "sable_autotune_cache_clear", "sable_plan_set_spmm_cols", "sable_plan_update_values",
    "sable_plan_set_spmm_depth", "sable_plan_device_error", "sable_probe_bulk_gather", "sable_set_wait_limit",
    "sable_get_wait_limit", "sable_probe_wait_limit", "sable_debug_fail_allocations",
    "sable_plan_set_inspector", "sable_debug_set_csr_column",
]

NFEAT = 24


class MlpShape(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_h1", ctypes.c_int32), ("n_h2", ctypes.c_int32),
                ("n_out", ctypes.c_int32)]


class SableError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("a_min", ctypes.c_int64), ("l_seg", ctypes.c_int32),
                ("w_max", ctypes.c_int32), ("d_max", ctypes.c_int64), ("count_min", ctypes.c_int64),
                ("coverage_min", ctypes.c_double), ("max_span", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("passes", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "m", "n", "nnz", "nnz_vdia", "nnz_vbr", "nnz_csr", "n_segments", "n_diagonals",
        "vdia_cells", "n_blocks", "vbr_cells", "n_items", "spmv_bytes", "csr_spmv_bytes")]


_lib = None


def lib():
    """Load libsable.so (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsable.so not built ({LIB_PATH}); run "
                               "paper_2407_00829_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "sable_default_params": ([i32, p], None),
            "sable_plan_create": ([i64, i64, i64, p, p, p, p], i32),
            "sable_plan_add_extractor": ([p, i32, p], i32),
            "sable_extract": ([p], i32),
            "sable_plan_set_inspector": ([p, i32], i32),
            "sable_debug_set_csr_column": ([p, i64, i32], i32),
            "sable_plan_upload": ([p, p], i32),
            "sable_spmv": ([p, p, p, p], i32),
            "sable_csr_spmv": ([p, p, p, p], i32),
            "sable_spmm": ([p, p, i64, i64, p, i64, i32, p], i32),
            "sable_csr_spmm": ([p, p, i64, i64, p, i64, p], i32),
            "sable_plan_info": ([p, p], i32),
            "sable_plan_get_segments": ([p, p], i32),
            "sable_plan_get_blocks": ([p, p], i32),
            "sable_plan_get_vdia_values": ([p, p], i32),
            "sable_plan_get_vbr_values": ([p, p], i32),
            "sable_plan_get_csr": ([p, p, p, p], i32),
            "sable_plan_set_tiling": ([p, i32, i64], i32),
            "sable_plan_status": ([p], i32),
            "sable_plan_destroy": ([p], i32),
            "sable_status_string": ([i32], ctypes.c_char_p),
            "sable_probe_gather": ([p, i64, i64, p, p], i32),
            "sable_probe_row_gather": ([p, i64, i64, i32, i64, p, p], i32),
            "sable_batch_create": ([p, i32, p], i32),
            "sable_batch_spmv": ([p, p, p, p], i32),
            "sable_batch_spmm": ([p, p, i64, p, i32, p], i32),
            "sable_batch_graph_spmv": ([p, p, p, p], i32),
            "sable_batch_graph_spmm": ([p, p, i64, p, i32, p], i32),
            "sable_graph_launch": ([p, p], i32),
            "sable_graph_destroy": ([p], i32),
            "sable_batch_status": ([p, p], i32),
            "sable_batch_destroy": ([p], i32),
            "sable_features_workspace_bytes": ([i64, i64, i64], i64),
            "sable_features": ([i64, i64, i64, p, p, p, i64, p, p], i32),
            "sable_plan_add_regions": ([p, i32, p, i64], i32),
            "sable_plan_get_region_stages": ([p, p, p], i32),
            "sable_plan_reset": ([p], i32),
            "sable_plan_get_tiling": ([p, p], i32),
            "sable_autotune": ([p, i32, i64, p, p, i32, i32, p, p, p], i32),
            "sable_autotune_cache_clear": ([], i64),
            "sable_probe_bulk_gather": ([p, i64, i64, p, p, p], i32),
            "sable_set_wait_limit": ([i64], i32),
            "sable_get_wait_limit": ([], i64),
            "sable_probe_wait_limit": ([p, p], i32),
            "sable_debug_fail_allocations": ([i64], None),
            "sable_plan_set_spmm_cols": ([p, i32], i32),
            "sable_plan_update_values": ([p, p, p], i32),
            "sable_plan_set_spmm_depth": ([p, i32], i32),
            "sable_plan_device_error": ([p, p], i32),
            "sable_error_workspace_bytes": ([], i64),
            "sable_error_norms": ([p, p, i64, p, p, i64, p], i32),
            "sable_mlp_param_count": ([p], i64),
            "sable_mlp_work_floats": ([p, i64], i64),
            "sable_mlp_forward": ([p, p, p, i64, p, p, p], i32),
            "sable_mlp_grad": ([p, p, p, p, p, i64, p, p, p, p], i32),
            "sable_mlp_adam": ([i64, p, p, p, p, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, p], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise SableError(st, what)


def default_params(kind: int) -> Params:
    p = Params()
    lib().sable_default_params(kind, ctypes.byref(p))
    return p


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int:
    return t.data_ptr()


class Tiling(ctypes.Structure):
    _fields_ = [("spmv_rows", ctypes.c_int32), ("spmv_bytes", ctypes.c_int64), ("spmm_cols", ctypes.c_int32),
                ("spmm_depth", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TUNE_SPMV, TUNE_SPMM_FP32, TUNE_SPMM_BF16, TUNE_SPMM_FP32_SPLIT, TUNE_CSR_SPMV = 0, 1, 2, 3, 4


class Plan:
    """A matrix, its ordered extractors and, after ``extract``/``upload``, its
    hybrid VDIA+VBR+CSR form on the host and the device."""

    def __init__(self, m: int, n: int, row, col, val):
        row = np.ascontiguousarray(row, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float32)
        if not (row.shape == col.shape == val.shape):
            raise ValueError("COO arrays differ in length")
        h = ctypes.c_void_p()
        _check(lib().sable_plan_create(int(m), int(n), int(val.size), row.ctypes.data,
                                       col.ctypes.data, val.ctypes.data, ctypes.byref(h)),
               "sable_plan_create")
        self._h = h
        self.m, self.n = int(m), int(n)
        self._stages = []

    # -- life cycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sable_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def add_extractor(self, kind: int, params: Optional[Params] = None, **kw):
        p = params if params is not None else default_params(kind)
        for k, v in kw.items():
            setattr(p, k, v)
        _check(lib().sable_plan_add_extractor(self._h, kind, ctypes.byref(p)), "add_extractor")
        self._stages.extend([kind] * max(1, p.passes))   # a multi-pass band extractor adds one stage per pass
        return self

    def add_regions(self, kind: int, regions):
        """A stage of given regions (k x 4 int64: VDIA (row0, nrows, off_lo,
        ndiag) or VBR (row0, nrows, col0, ncols)) in place of a search."""
        g = np.ascontiguousarray(np.asarray(regions, dtype=np.int64).reshape(-1, 4))
        _check(lib().sable_plan_add_regions(self._h, kind, g.ctypes.data, g.shape[0]), "add_regions")
        self._stages.append(kind)
        return self

    def update_values(self, val, stream=None):
        """Same structure, new values (the COO order given at creation)."""
        v = np.ascontiguousarray(val, dtype=np.float32)
        if stream is None:   # a plan that was never uploaded needs no stream (nor a GPU)
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        _check(lib().sable_plan_update_values(self._h, v.ctypes.data if v.size else None, _stream_handle(stream)),
               "sable_plan_update_values")
        return self

    def reset(self):
        """Drop stages, extraction and device tables; keep the matrix."""
        _check(lib().sable_plan_reset(self._h), "sable_plan_reset")
        self._stages = []
        return self

    def region_stages(self):
        info = self.info()
        ss = np.zeros(max(1, info["n_segments"]), dtype=np.int32)
        bs = np.zeros(max(1, info["n_blocks"]), dtype=np.int32)
        _check(lib().sable_plan_get_region_stages(self._h, ss.ctypes.data, bs.ctypes.data), "get_region_stages")
        return ss[:info["n_segments"]], bs[:info["n_blocks"]]

    def region_table(self):
        """The extracted plan as stages [(kind, regions k x 4)]: VDIA / VBR
        stages carry their regions, CSR stages none.  ``add_stages`` on a plan
        of the same matrix rebuilds this extraction without searching."""
        ss, bs = self.region_stages()
        segs, blks = self.segments(), self.blocks()
        out = []
        for t, kind in enumerate(self._stages):
            if kind == VDIA:
                out.append((kind, segs[ss == t]))
            elif kind == VBR:
                out.append((kind, blks[bs == t]))
            else:
                out.append((kind, np.zeros((0, 4), np.int64)))
        return out

    def add_stages(self, table):
        for kind, regions in table:
            if kind == CSR:
                self.add_extractor(CSR)
            else:
                self.add_regions(kind, regions)
        return self

    def set_inspector(self, where: int):
        """INSPECT_HOST (default) or INSPECT_DEVICE: where sable_extract runs the
        extractors' counting steps (same regions either way)."""
        _check(lib().sable_plan_set_inspector(self._h, where), "sable_plan_set_inspector")
        return self

    def extract(self):
        _check(lib().sable_extract(self._h), "sable_extract")
        return self

    def set_tiling(self, spmv_rows=512, spmv_bytes=48 * 1024, spmm_cols=None, spmm_depth=None):
        _check(lib().sable_plan_set_tiling(self._h, spmv_rows, spmv_bytes), "set_tiling")
        if spmm_cols is not None:
            _check(lib().sable_plan_set_spmm_cols(self._h, spmm_cols), "set_spmm_cols")
        if spmm_depth is not None:
            _check(lib().sable_plan_set_spmm_depth(self._h, spmm_depth), "set_spmm_depth")
        return self

    def upload(self, stream=None):
        _check(lib().sable_plan_upload(self._h, _stream_handle(stream)), "sable_plan_upload")
        return self

    # -- compute (device tensors)
    def spmv(self, x, y, stream=None):
        _check(lib().sable_spmv(self._h, _dptr(x), _dptr(y), _stream_handle(stream)), "sable_spmv")
        return y

    def csr_spmv(self, x, y, stream=None):
        _check(lib().sable_csr_spmv(self._h, _dptr(x), _dptr(y), _stream_handle(stream)), "sable_csr_spmv")
        return y

    def spmm(self, B, C, precision: int = FP32, stream=None):
        N = B.shape[1]
        _check(lib().sable_spmm(self._h, _dptr(B), N, B.stride(0), _dptr(C), C.stride(0), precision,
                                _stream_handle(stream)), "sable_spmm")
        return C

    def csr_spmm(self, B, C, stream=None):
        N = B.shape[1]
        _check(lib().sable_csr_spmm(self._h, _dptr(B), N, B.stride(0), _dptr(C), C.stride(0),
                                    _stream_handle(stream)), "sable_csr_spmm")
        return C

    # -- host views
    def info(self) -> dict:
        s = Stats()
        _check(lib().sable_plan_info(self._h, ctypes.byref(s)), "sable_plan_info")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def segments(self) -> np.ndarray:
        k = self.info()["n_segments"]
        out = np.zeros((k, 4), dtype=np.int64)
        _check(lib().sable_plan_get_segments(self._h, out.ctypes.data), "get_segments")
        return out

    def blocks(self) -> np.ndarray:
        k = self.info()["n_blocks"]
        out = np.zeros((k, 4), dtype=np.int64)
        _check(lib().sable_plan_get_blocks(self._h, out.ctypes.data), "get_blocks")
        return out

    def vdia_values(self) -> np.ndarray:
        out = np.zeros(self.info()["vdia_cells"], dtype=np.float32)
        _check(lib().sable_plan_get_vdia_values(self._h, out.ctypes.data), "get_vdia_values")
        return out

    def vbr_values(self) -> np.ndarray:
        out = np.zeros(self.info()["vbr_cells"], dtype=np.float32)
        _check(lib().sable_plan_get_vbr_values(self._h, out.ctypes.data), "get_vbr_values")
        return out

    def csr(self):
        k = self.info()["nnz_csr"]
        rp = np.zeros(self.m + 1, dtype=np.int64)
        ci = np.zeros(max(k, 1), dtype=np.int32)
        cv = np.zeros(max(k, 1), dtype=np.float32)
        _check(lib().sable_plan_get_csr(self._h, rp.ctypes.data, ci.ctypes.data, cv.ctypes.data), "get_csr")
        return rp, ci[:k], cv[:k]

    def status(self) -> int:
        return lib().sable_plan_status(self._h)

    def device_error(self):
        """[status, check tag, index, bound] recorded by the plan's kernels
        (see sable_plan_device_error)."""
        out = (ctypes.c_int32 * 4)()
        _check(lib().sable_plan_device_error(self._h, out), "sable_plan_device_error")
        return list(out)

    def debug_set_csr_column(self, entry: int, value: int):
        """Debug build only: overwrite one device CSR remainder column."""
        _check(lib().sable_debug_set_csr_column(self._h, int(entry), int(value)), "sable_debug_set_csr_column")
        return self

    def tiling(self) -> dict:
        t = Tiling()
        _check(lib().sable_plan_get_tiling(self._h, ctypes.byref(t)), "get_tiling")
        return t.as_dict()

    def autotune(self, op: int, inp, out, reps: int = 10, use_cache: bool = True, stream=None):
        """Pick and apply the fastest tiling for op (TUNE_SPMV / TUNE_CSR_SPMV /
        TUNE_SPMM_FP32 / TUNE_SPMM_BF16 / TUNE_SPMM_FP32_SPLIT) by timing it on
        the device; returns (tiling, ms)."""
        N = 0 if op in (TUNE_SPMV, TUNE_CSR_SPMV) else inp.shape[1]
        t = Tiling()
        ms = ctypes.c_float()
        _check(lib().sable_autotune(self._h, op, N, _dptr(inp), _dptr(out), reps, int(use_cache), ctypes.byref(t),
                                    ctypes.byref(ms), _stream_handle(stream)), "sable_autotune")
        return t.as_dict(), ms.value


def autotune_cache_clear() -> int:
    return lib().sable_autotune_cache_clear()


def error_norms(y, ref, stream=None):
    """FP64 device reduction of an FP32 result y against an FP64 reference
    (both device tensors, same number of elements).  Returns a dict with
    max_abs_err, max_abs_ref, sq_err, sq_ref, normwise (max_abs_err /
    max_abs_ref) and rel2 (sqrt(sq_err / sq_ref))."""
    import torch
    if y.dtype != torch.float32 or ref.dtype != torch.float64 or y.numel() != ref.numel():
        raise ValueError("y must be float32 and ref float64 with as many elements")
    y, ref = y.contiguous(), ref.contiguous()
    wb = lib().sable_error_workspace_bytes()
    work = torch.empty(wb, dtype=torch.uint8, device=y.device)
    out = torch.empty(4, dtype=torch.float64, device=y.device)
    _check(lib().sable_error_norms(_dptr(y), _dptr(ref), y.numel(), _dptr(out), _dptr(work), wb,
                                   _stream_handle(stream)), "sable_error_norms")
    e, r, e2, r2 = out.cpu().tolist()
    nw = e / r if r > 0 else (0.0 if e == 0 else float("inf"))
    return {"max_abs_err": e, "max_abs_ref": r, "sq_err": e2, "sq_ref": r2, "normwise": nw,
            "rel2": math.sqrt(e2 / r2) if r2 > 0 else (0.0 if e2 == 0 else float("inf"))}


def save_region_table(path, table, m: int, n: int, nnz: int):
    """Write a region table (``Plan.region_table()``) to an .npz file."""
    arrs = {f"stage{t}": np.asarray(g, np.int64) for t, (_, g) in enumerate(table)}
    np.savez(path, kinds=np.array([k for k, _ in table], np.int32), shape=np.array([m, n, nnz], np.int64),
             **arrs)


def load_region_table(path):
    """Read a region table: ([(kind, regions)], (m, n, nnz))."""
    d = np.load(path)
    kinds = d["kinds"].tolist()
    return [(k, d[f"stage{t}"]) for t, k in enumerate(kinds)], tuple(int(v) for v in d["shape"])


def probe_gather(x, count: int, out, stream=None):
    """Launch the random-gather calibration kernel (see include/sable.h)."""
    _check(lib().sable_probe_gather(_dptr(x), x.numel(), int(count), _dptr(out), _stream_handle(stream)),
           "sable_probe_gather")


def probe_bulk_gather(x, count: int, out, status, stream=None):
    """Launch the bulk-copy random-gather calibration kernel (see include/sable.h);
    ``status`` is a device int32 tensor of one element."""
    _check(lib().sable_probe_bulk_gather(_dptr(x), x.numel(), int(count), _dptr(out), _dptr(status),
                                         _stream_handle(stream)), "sable_probe_bulk_gather")


def set_wait_limit(cycles: int):
    """Budget in GPU clock cycles of every bounded device wait (process-wide)."""
    _check(lib().sable_set_wait_limit(int(cycles)), "sable_set_wait_limit")


def wait_limit() -> int:
    return int(lib().sable_get_wait_limit())


def probe_wait_limit(status, stream=None):
    """A bounded wait nothing satisfies; ``status`` (device int32) gets the outcome."""
    _check(lib().sable_probe_wait_limit(_dptr(status), _stream_handle(stream)), "sable_probe_wait_limit")


def probe_row_gather(B, count: int, out, stream=None):
    """Launch the random row-gather calibration kernel on a 2-D float32 B
    (see include/sable.h)."""
    if B.dim() != 2 or B.stride(1) != 1:
        raise ValueError("B must be a row-major 2-D tensor")
    _check(lib().sable_probe_row_gather(_dptr(B), B.shape[0], B.stride(0), B.shape[1], int(count), _dptr(out),
                                        _stream_handle(stream)), "sable_probe_row_gather")


class Graph:
    """A captured CUDA graph of batch launches (keeps its operand tables alive)."""

    def __init__(self, handle, keep):
        self._h, self._keep = handle, keep

    def launch(self, stream=None):
        _check(lib().sable_graph_launch(self._h, _stream_handle(stream)), "sable_graph_launch")

    def close(self):
        if self._h is not None and self._h.value:
            lib().sable_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many uploaded plans computed by one grouped launch per op."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * max(1, len(self.plans)))(*[P.handle for P in self.plans])
        h = ctypes.c_void_p()
        _check(lib().sable_batch_create(arr, len(self.plans), ctypes.byref(h)), "sable_batch_create")
        self._h = h

    @staticmethod
    def _ptrs(tensors):
        import torch
        dev = tensors[0].device if tensors else torch.device("cuda")
        return torch.tensor([t.data_ptr() for t in tensors] or [0], dtype=torch.int64, device=dev)

    def spmv(self, xs, ys, stream=None):
        px, py = self._ptrs(xs), self._ptrs(ys)
        _check(lib().sable_batch_spmv(self._h, px.data_ptr(), py.data_ptr(), _stream_handle(stream)),
               "sable_batch_spmv")
        return (px, py)

    def spmm(self, Bs, Cs, N, precision=FP32, stream=None):
        pb, pc = self._ptrs(Bs), self._ptrs(Cs)
        _check(lib().sable_batch_spmm(self._h, pb.data_ptr(), int(N), pc.data_ptr(), precision,
                                      _stream_handle(stream)), "sable_batch_spmm")
        return (pb, pc)

    def graph_spmv(self, xs, ys) -> Graph:
        px, py = self._ptrs(xs), self._ptrs(ys)
        import torch
        torch.cuda.synchronize()
        g = ctypes.c_void_p()
        _check(lib().sable_batch_graph_spmv(self._h, px.data_ptr(), py.data_ptr(), ctypes.byref(g)),
               "sable_batch_graph_spmv")
        return Graph(g, (px, py, xs, ys))

    def graph_spmm(self, Bs, Cs, N, precision=FP32) -> Graph:
        pb, pc = self._ptrs(Bs), self._ptrs(Cs)
        import torch
        torch.cuda.synchronize()
        g = ctypes.c_void_p()
        _check(lib().sable_batch_graph_spmm(self._h, pb.data_ptr(), int(N), pc.data_ptr(), precision,
                                            ctypes.byref(g)), "sable_batch_graph_spmm")
        return Graph(g, (pb, pc, Bs, Cs))

    def device_error(self) -> int:
        v = ctypes.c_int32()
        _check(lib().sable_batch_status(self._h, ctypes.byref(v)), "sable_batch_status")
        return v.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sable_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(m, n, row, col, stream=None):
    """SABLE_NFEAT structural features of a COO matrix given as device int32
    tensors (computed by the library's feature kernels); returns a device tensor."""
    import torch
    nnz = row.numel()
    wb = lib().sable_features_workspace_bytes(int(m), int(n), int(nnz))
    work = torch.empty(max(wb, 16), dtype=torch.uint8, device=row.device)
    out = torch.empty(NFEAT, dtype=torch.float32, device=row.device)
    _check(lib().sable_features(int(m), int(n), int(nnz), _dptr(row), _dptr(col), _dptr(work), wb, _dptr(out),
                                _stream_handle(stream)), "sable_features")
    return out


class Mlp:
    """Device MLP n_in -> h1 -> h2 -> n_out (ReLU, ReLU, linear) trained with the
    library's kernels; parameters / Adam state are torch device tensors."""

    def __init__(self, n_in, h1, h2, n_out, seed=0, device="cuda"):
        import torch
        self.shape = MlpShape(n_in, h1, h2, n_out)
        self.count = lib().sable_mlp_param_count(ctypes.byref(self.shape))
        rng = np.random.default_rng(seed)
        parts = []
        for a, b in ((n_in, h1), (h1, h2), (h2, n_out)):
            parts.append(rng.standard_normal((a, b)) * np.sqrt(2.0 / a))
            parts.append(np.zeros(b))
        flat = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
        assert flat.size == self.count
        self.params = torch.from_numpy(flat).to(device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._work = {}

    def _w(self, batch):
        import torch
        if batch not in self._work:
            n = lib().sable_mlp_work_floats(ctypes.byref(self.shape), int(batch))
            self._work[batch] = torch.empty(n, dtype=torch.float32, device=self.params.device)
        return self._work[batch]

    def forward(self, X, stream=None):
        import torch
        B = X.shape[0]
        Y = torch.empty(B, self.shape.n_out, dtype=torch.float32, device=X.device)
        _check(lib().sable_mlp_forward(ctypes.byref(self.shape), _dptr(self.params), _dptr(X), B, _dptr(Y),
                                       _dptr(self._w(B)), _stream_handle(stream)), "sable_mlp_forward")
        return Y

    def grad(self, X, T, mask=None, stream=None):
        import torch
        B = X.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        _check(lib().sable_mlp_grad(ctypes.byref(self.shape), _dptr(self.params), _dptr(X), _dptr(T),
                                    _dptr(mask) if mask is not None else None, B, _dptr(self.grads),
                                    _dptr(loss), _dptr(self._w(B)), _stream_handle(stream)), "sable_mlp_grad")
        return loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        _check(lib().sable_mlp_adam(self.count, _dptr(self.params), _dptr(self.grads), _dptr(self.m), _dptr(self.v),
                                    self.step, lr, beta1, beta2, eps, _stream_handle(stream)), "sable_mlp_adam")


def plan_from(A: dict, extractors, tiling: Optional[dict] = None, upload: bool = True, stream=None,
              inspector: int = INSPECT_HOST) -> Plan:
    """Create, extract and (optionally) upload a plan for a COO dict
    {m, n, row, col, val}; ``extractors`` is a list of (kind, params-dict or None)."""
    P = Plan(A["m"], A["n"], A["row"], A["col"], A["val"])
    for kind, kw in extractors:
        P.add_extractor(kind, **(kw or {}))
    if inspector != INSPECT_HOST:
        P.set_inspector(inspector)
    P.extract()
    if tiling:
        P.set_tiling(**tiling)
    if upload:
        P.upload(stream)
    return P
