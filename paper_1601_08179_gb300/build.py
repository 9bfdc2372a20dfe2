"""Builds libsemgb.so (the C-ABI library of include/sem.h) for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into a shared library next to this file.  `build(debug=True)` (or
--debug) builds libsemgb_debug.so instead, compiled with SEM_DEBUG: every
kernel checks the skeleton entity offsets and class indices it forms before
any access and keeps a record of failures (sem_debug_oob in include/sem.h);
the binding loads it when SEM_LIB names it.  Usage:

    python -m paper_1601_08179_gb300.build [--force] [--debug]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsemgb.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libsemgb_debug.so")
SOURCES = ["sem_host.cpp", "sem_kernels.cu", "sem_apply.cu", "sem_apply_plane.cu", "sem_apply_slab.cu",
           "sem_apply_elem.cu", "sem_apply_row.cu", "sem_apply_pencil.cu", "sem_compare.cu", "sem_api.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(debug: bool = False):
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", os.path.join(HERE, "..", "include")]
    return f + (["-DSEM_DEBUG"] if debug else [])


def _compile(src: str, debug: bool = False) -> str:
    obj = os.path.join(BUILD_DEBUG if debug else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *_flags(debug), "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "sem.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD_DEBUG if debug else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda src: _compile(src, debug), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), ARCH, "-shared", "-o", tmp, *objs, "-lcublas"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv))
