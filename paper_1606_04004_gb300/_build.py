"""Builds libprunedq.so in-tree with nvcc for sm_103a (one -gencode, one
translation unit per source file, compiled in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libprunedq.so")
LIB_CHECKED = os.path.join(HERE, "libprunedq_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "--expt-relaxed-constexpr"]
SOURCES = ["basis.cpp", "lattice.cu", "apply_h.cu", "krylov.cu", "capi.cu", "noalloc.cu", "adjoint.cu", "pvb.cu", "peaks.cu", "tc_fibre.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libprunedq")


def _compile(src: str, debug: bool = False) -> str:
    obj = os.path.join(BUILD_DIR, src + (".dbg.o" if debug else ".o"))
    flags = NVCC_FLAGS + (["-DPQ_BOUNDS_CHECK"] if debug else [])
    cmd = [_nvcc(), *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-x", "cu", *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "prunedq.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build_library(force: bool = False, debug: bool = False) -> str:
    """Build libprunedq.so (or, with debug=True, the self-checking
    libprunedq_checked.so whose kernels record out-of-range indices instead
    of accessing them)."""
    lib = LIB_CHECKED if debug else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda f: _compile(f, debug), SOURCES))
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
           "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib
