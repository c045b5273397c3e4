"""Builds libgrnnd.so (the CUDA library behind include/grnnd.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2510_02774_gb300/_build/libgrnnd.so``.  Run ``python -m paper_2510_02774_gb300.build``.
``build(checks=True)`` makes the checked variant in ``_build_checks/`` (-DGRNND_CHECKS=1:
device bounds checks that report through the step's status word instead of faulting; the
stand-in for a memory checker, which this pool does not run).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libgrnnd.so")
OUT_CHECKS = os.path.join(PKG, "_build_checks")
LIB_CHECKS = os.path.join(OUT_CHECKS, "libgrnnd.so")
UNITS = ["pool_kernels.cu", "wide_kernels.cu", "search_kernels.cu", "capi.cu", "noalloc.cu", "server.cu"]
HEADERS = ["common.cuh", "internal.h", "kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", SRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "grnnd.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checks: bool = False) -> str:
    out = OUT_CHECKS if checks else OUT
    lib = LIB_CHECKS if checks else LIB
    extra = (*extra, "-DGRNND_CHECKS=1") if checks else tuple(extra)
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(out, u.replace(".cu", ".o"))
        if force or _stale(obj, src):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}")

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out, u.replace(".cu", ".o")) for u in UNITS]
    if jobs or force or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
