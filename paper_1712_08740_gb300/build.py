"""Builds libhelm.so (the CUDA library behind include/helm.h) in-tree.

Every translation unit is compiled for sm_103a (GB300) only, in parallel,
then linked into ``paper_1712_08740_gb300/lib/libhelm.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libhelm.so")
SOURCES = ["setup.cu", "stencil.cu", "stencil_ds.cu", "vfused.cu", "vfused_f64.cu", "vfused_mixed.cu", "vfused_c64.cu", "vfused_ds.cu", "coarse.cu", "coarse_tc.cu", "krylov.cu", "krylov_ds.cu", "krylov_c64.cu", "cycle.cu", "api.cu", "fgmres.cu", "noalloc.cu", "serve.cu", "tune.cu", "block.cu", "recycle.cu"]
HEADERS = ["helm_internal.cuh", "vfused.cuh", "grid.cuh", "vcycle.cuh", "cycle.cuh", "pipe.cuh", "tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhelm")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "helm.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def _is_native_lib() -> bool:
    """The library was built for this machine's architecture."""
    try:
        with open(LIB, "rb") as fh:
            head = fh.read(20)
    except OSError:
        return False
    import platform
    mach = int.from_bytes(head[18:20], "little")
    want = {"x86_64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine())
    return want is None or mach == want


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libhelm.so if it is missing, stale or foreign; return its path."""
    if not force and not _stale() and _is_native_lib():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
