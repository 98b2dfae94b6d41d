"""Builds libsexpm.so in-tree with nvcc for sm_103a (GB300).

Usage: ``python -m paper_2110_04493_gb300.build`` or ``build()`` from Python.
Each translation unit is compiled in parallel; the shared library links the
CUDA runtime statically and has no PyTorch dependency.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsexpm.so")
SOURCES = ["api.cu", "kernels_spgemm.cu", "kernels_csr.cu", "kernels_filter.cu", "kernels_adjoint.cu", "kernels_spmm.cu",
           "batched_graph.cu", "complex_path.cu",
           "noalloc.cu", "plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
            *ARCH, *extra]


def _compile(src: str, extra) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, *_flags(extra)]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-Xcompiler",
               "-fPIC", "-I", os.path.join(ROOT, "include")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sexpm.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every CUDA/C++ source and link libsexpm.so; returns its path.

    SEXPM_NVCC_FLAGS (environment) adds nvcc flags, e.g. -D overrides of tuning constants."""
    extra = tuple(extra) + tuple(os.environ.get("SEXPM_NVCC_FLAGS", "").split())
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), "-shared", "-o", tmp, *objs, *ARCH]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
