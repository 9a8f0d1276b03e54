"""Builds libpairgal.so in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked with the shared CUDA runtime so that the library and PyTorch share
one runtime instance. The files that decide integers from floating point
(pair bins, mesh nodes, Q32.32 weights) are compiled with -fmad=false.

    python -m paper_1705_03464_gb300.build_lib
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpairgal.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
NO_FMA = {"pg_pairs.cu", "pg_mesh.cu"}
# the longest compiles first, so the parallel build ends with the short ones
SOURCES = ["pg_fft_z_f32.cu", "pg_fft_f32.cu", "pg_fft_z_f64.cu", "pg_fft_f64.cu", "pg_api.cu",
           "pg_pairs.cu", "pg_mesh.cu", "pg_scan.cu", "pg_bin.cu", "pg_tma.cu", "pg_noalloc.cu",
           "pg_adjoint.cu", "pg_batch.cu", "pg_smooth.cu", "pg_smooth_adj.cu", "pg_hod.cu"]


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpairgal")


def _compile(nvcc, src):
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc, *ARCH, *COMMON]
    if src in NO_FMA:
        cmd.append("-fmad=false")
    cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    for f in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    hdr = os.path.join(os.path.dirname(HERE), "include", "pairgal.h")
    return os.path.exists(hdr) and os.path.getmtime(hdr) > t


def build(force: bool = False, verbose: bool = True) -> str:
    if not force and not _stale():
        return OUT
    import fcntl
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)   # one builder at a time (pytest, bench ranks)
        if not force and not _stale():
            return OUT
        return _build_locked(verbose)


def _build_locked(verbose: bool) -> str:
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print(f"built {OUT}", file=sys.stderr)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv)
