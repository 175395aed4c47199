"""Build libsable.so in-tree: nvcc for the CUDA units (sm_103a only), g++ for
the host units, compiled in parallel and linked into
``paper_2407_00829_gb300/_build/libsable.so``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsable.so")
# the debug build: the same sources with SABLE_CHECKS (index checks in the hot
# kernels that record a bad column in the plan's device error word)
OUT_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(OUT_CHECKS, "libsable.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}"] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-pthread", "-fno-fast-math", "-ffp-contract=off",
             f"-I{INCLUDE}"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(SRC) if f.endswith(".cpp"))
    hdr = sorted(f for f in os.listdir(SRC) if f.endswith(".h"))
    return cu, cpp, hdr


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    cu, cpp, hdr = sources()
    deps = [os.path.join(SRC, f) for f in cu + cpp + hdr] + [os.path.join(INCLUDE, "sable.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Build libsable.so (checks=True: the debug build with index checks, in
    _build_checks/) if any source is newer; returns its path."""
    out, lib = (OUT_CHECKS, LIB_CHECKS) if checks else (OUT, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp, _ = sources()
    extra = ["-DSABLE_CHECKS"] if checks else []
    jobs = []
    for f in cu:
        o = os.path.join(out, f + ".o")
        jobs.append(([nvcc] + NVCC_FLAGS + extra + ["-c", os.path.join(SRC, f), "-o", o], o))
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")   # NVTX header
    for f in cpp:
        o = os.path.join(out, f + ".o")
        jobs.append((["g++"] + CXX_FLAGS + extra + [f"-I{cuda_inc}", "-c", os.path.join(SRC, f), "-o", o], o))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        list(ex.map(run, [j[0] for j in jobs]))
    tmp = lib + f".{os.getpid()}.tmp"
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + [j[1] for j in jobs] + ["-lpthread"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checks="--checks" in sys.argv))
