"""Build libpdmk.so (sm_103a) in-tree with nvcc.  Used by __graft_entry__.build()."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpdmk.so")
SOURCES = ["capi.cu", "pw.cu", "gpu_build.cu", "host_plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newest_input():
    t = 0.0
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    t = max(t, os.path.getmtime(os.path.join(ROOT, "include", "pdmk.h")))
    return t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    cmd = ["nvcc", "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3,-fopenmp",
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-shared", "-o", LIB]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    cmd += ["-lcufft", "-lgomp"]  # OpenMP: the host planner's per-point and per-box loops
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
