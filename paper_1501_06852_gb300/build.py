"""Builds libpfc.so (the CUDA stage solver) in-tree for sm_103a with nvcc.

Usage: ``python -m paper_1501_06852_gb300.build`` or ``build()`` from Python.
The translation units compile in parallel; the shared library lands in
``paper_1501_06852_gb300/_lib/libpfc.so`` (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libpfc.so")
SOURCES = ["api.cu", "solver.cu", "kernels.cu", "noalloc.cu", "host_mesh.cpp", "refelem.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpfc.so")
    return cand


def _flags(verbose: bool) -> list[str]:
    f = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-I", CSRC,
         "-I", os.path.join(ROOT, "include"), "-Xcompiler", "-fPIC,-fopenmp,-O3"] + ARCH
    # extra preprocessor definitions, e.g. PFC_NVCC_DEFINES="PFC_SOLVER_THREADS=1024 PFC_SPMV_WIDE=1"
    f += ["-D" + d for d in os.environ.get("PFC_NVCC_DEFINES", "").split() if d]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pfc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source for sm_103a and link libpfc.so; returns its path."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose)
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj] + _flags(False)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lgomp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
