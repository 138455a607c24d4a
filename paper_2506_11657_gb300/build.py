"""Build the TEM C-ABI library (libtem.so) in-tree for sm_103a.

Every translation unit compiles in parallel with nvcc at -O3 (-gencode
arch=compute_103a,code=sm_103a -lineinfo); the objects link into
``paper_2506_11657_gb300/libtem.so`` next to this file.  No cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libtem.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["grid.cu", "solver.cu", "forward.cu", "serve.cu", "noalloc.cu", "geometry.cpp", "poles.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtem.so")
    return cand


def _compile(src, nvcc, extra):
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *extra, "-c", path, "-o", obj]
    else:
        cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *extra, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra=(), out=None, build_dir=None) -> str:
    """Compile and link; returns the library path.  Rebuilds only when a source is newer."""
    global BUILD, OUT
    if out is not None or build_dir is not None:
        saved = (BUILD, OUT)
        BUILD, OUT = build_dir or BUILD, out or OUT
        try:
            return build(verbose, extra)
        finally:
            BUILD, OUT = saved
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "tem.h")]
    if os.path.exists(OUT) and all(os.path.getmtime(d) <= os.path.getmtime(OUT) for d in deps):
        return OUT
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, list(extra)), srcs))
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print("built", OUT, file=sys.stderr)
    return OUT


def build_checked(verbose: bool = False) -> str:
    """The bounds-checked variant (-DTEM_CHECK_BOUNDS: every global index and TMA box start of the
    hot kernels is checked; a failing check is recorded and reported instead of faulting) as
    libtem_checked.so next to libtem.so.  Select it at run time with TEM_LIB=<path>."""
    return build(verbose, extra=("-DTEM_CHECK_BOUNDS",), out=os.path.join(HERE, "libtem_checked.so"),
                 build_dir=os.path.join(HERE, "_build_checked"))


if __name__ == "__main__":
    print(build(verbose=True))
