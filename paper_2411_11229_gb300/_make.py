"""Compile libhweno.so (the CUDA library behind include/hweno.h) for sm_103a, in-tree."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libhweno.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
SOURCES = ["hweno_api.cu", "hweno_batch.cu", "hweno_adjoint.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the HWENO CUDA library cannot be built")


LIB_BOUNDS = os.path.join(PKG, "libhweno_bounds.so")


def lib_path(bounds_check: bool = False) -> str:
    return LIB_BOUNDS if bounds_check else LIB


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "hweno.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Build (if stale) and return the path of libhweno.so, or with bounds_check of
    libhweno_bounds.so: the same sources compiled with -DHWENO_BOUNDS_CHECK, whose kernels check
    every index they form (a debugging aid; see hweno_bounds_status in include/hweno.h)."""
    lib = lib_path(bounds_check)
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    objdir = os.path.join(PKG, "_build_bounds" if bounds_check else "_build")
    os.makedirs(objdir, exist_ok=True)
    defs = ["-DHWENO_BOUNDS_CHECK"] if bounds_check else []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-I", os.path.join(ROOT, "include"), "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, len(SOURCES))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> tuple:
    """Both libraries (libhweno.so and the bounds-checked libhweno_bounds.so), compiled
    concurrently."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force)
        b = ex.submit(build, force, False, True)
        return a.result(), b.result()


if __name__ == "__main__":
    print(build(force=True, verbose=True))
