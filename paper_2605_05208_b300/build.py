"""Builds libmdls.so in-tree from csrc/*.cu (and the host-only csrc/*.cpp) for sm_103a (B300)
with nvcc.

Usage: python -m paper_2605_05208_b300.build [--force] [--bounds]
--bounds builds libmdls_bounds.so instead: every device-side gather checks its index and a call
that met an index out of range returns MD_ERR_BOUNDS (select it with MDLS_LIBRARY=<path>).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmdls.so")
LIB_BOUNDS = os.path.join(HERE, "libmdls_bounds.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu"))) + sorted(glob.glob(os.path.join(CSRC, "*.cpp")))


def deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "mdls.h")]


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compiles every source and links libmdls.so (rebuilds only when a source is newer);
    bounds: the bounds-checked libmdls_bounds.so."""
    out = LIB_BOUNDS if bounds else LIB
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= t for d in deps()):
            return out
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "--fmad=false", "-I", INCLUDE, "-o", out, *sources(), "-lcudart"]
    if bounds:
        cmd.insert(1, "-DMD_DEBUG_BOUNDS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
