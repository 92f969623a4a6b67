"""Build libbege.so in-tree for sm_103a with nvcc (no cmake).

Translation units compile in parallel; the shared library links the CUDA
runtime statically.  Usage: ``python -m paper_1708_01609_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbege.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
          "-Xcompiler", "-fvisibility=hidden",
          "-I", os.path.join(HERE, "..", "include")]
SOURCES = ["bege_corr_tc.cu", "bege_corr_multi.cu", "bege_corr_s16.cu", "bege_corr_s8.cu", "bege_corr_s4.cu", "bege_corr_s2.cu",
           "bege_corr_s1.cu", "bege_segment_bank.cu", "bege_batch.cu", "bege_noalloc.cu", "bege_api.cpp",
           "bege_serve.cpp"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _compile(src: str, verbose_ptxas: bool) -> str:
    out = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, "-c", os.path.join(CSRC, src), "-o", out]
    if src.endswith(".cu"):
        cmd += ["-lineinfo"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return out


def _up_to_date() -> bool:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "bege.h"))
    if not os.path.exists(LIB):
        return False
    return os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in srcs + headers)


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile libbege.so if any source is newer than it.  Processes that
    build at the same time (one per rank) serialise on a lock file; the
    second finds the library up to date."""
    import fcntl
    os.makedirs(OBJ, exist_ok=True)
    if not force and _up_to_date():
        return LIB
    with open(os.path.join(OBJ, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and _up_to_date():
            return LIB
        return _build_locked(verbose_ptxas)


def _build_locked(verbose_ptxas: bool) -> str:
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
