"""Build libsynim.so (the sm_103a CUDA library behind include/synim.h) in-tree,
and its bounds-checked twin libsynim_bounds.so (-DSYNIM_DEBUG_BOUNDS: every
index of the IM kernels tested against its buffer; loaded instead of the
release library when SYNIM_DEBUG_BOUNDS=1 is set in the environment).

    python -m paper_2606_07759_b300.build [--force] [--bounds]

nvcc cross-compiles for compute_103a/sm_103a; no GPU is needed to build.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsynim.so")
LIB_BOUNDS = os.path.join(PKG, "libsynim_bounds.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-shared",
    "--cudart", "shared",
    "-Xlinker", "-rpath,/usr/local/cuda/lib64",
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def lib_path(bounds: bool = False) -> str:
    return LIB_BOUNDS if bounds else LIB


def stale(bounds: bool = False) -> bool:
    lib = lib_path(bounds)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    lib = lib_path(bounds)
    if not force and not stale(bounds):
        return lib
    flags = NVCC_FLAGS + (["-DSYNIM_DEBUG_BOUNDS"] if bounds else [])
    cmd = [NVCC, *flags, "-I", INCLUDE, "-I", CSRC, "-o", lib + ".tmp", *sources()]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
