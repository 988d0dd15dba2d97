"""Build libstk.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit is compiled in parallel into ``_build/`` and linked into
``paper_1912_04753_gb300/_build/libstk.so``.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libstk.so")

SOURCES = ["index.cu", "pair.cu", "pair_setup.cpp", "stk.cu", "noalloc.cu", "serve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstk.so")


def _flags(verbose_ptx: bool) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "-I", INCLUDE, "-I", CSRC]
    if verbose_ptx:
        f += ["-Xptxas", "-v"]
    return f


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "stk.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose_ptx: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(path), hdr):
            jobs.append((path, obj))

    def compile_one(job):
        path, obj = job
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc] + _flags(verbose_ptx) + ["-c", path, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(path)}:\n{r.stdout}{r.stderr}")
        os.replace(tmp, obj)
        return r.stdout + r.stderr

    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(compile_one, jobs))
    stale = not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs)
    if jobs or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
        os.replace(tmp, LIB)
    if verbose_ptx:
        for lg in logs:
            sys.stdout.write(lg)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptx="-v" in sys.argv))
