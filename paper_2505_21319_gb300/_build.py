"""In-tree build of the CUDA library ``lib/libefunc.so`` (sm_103a only).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library with the CUDA runtime linked statically.  The
build is skipped when the library is newer than every source and header.

``build(debug=True)`` makes ``lib/libefunc_debug.so``: the same sources with
``-DEFUNC_DEBUG_BOUNDS``, whose kernels check the indices of their hot
gathers and scatters and record the first failing check (read with
``efunc_debug_bounds``); the binding loads it when ``EFUNC_DEBUG_BOUNDS=1``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libefunc.so")
LIB_DEBUG = os.path.join(LIBDIR, "libefunc_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def lib_path(debug: bool = False) -> str:
    return LIB_DEBUG if debug else LIB


def up_to_date(debug: bool = False) -> bool:
    lib = lib_path(debug)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link ``libefunc.so`` (``libefunc_debug.so`` with bounds
    checks when debug); returns its path."""
    LIB = lib_path(debug)
    if not force and up_to_date(debug):
        return LIB
    objdir = OBJDIR + ("_debug" if debug else "")
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    extra = ["-DEFUNC_DEBUG_BOUNDS"] if debug else []

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
