"""Builds the in-tree CUDA library ``libhram.so`` for B300 (sm_103a).

Run as ``python -m paper_2609_05494_b300.build`` or call :func:`build`.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "hram_capi.cu"), os.path.join(HERE, "csrc", "hram_persist.cu")]
DEPS = SRC + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                    glob.glob(os.path.join(HERE, "csrc", "*.h"))) + [os.path.join(ROOT, "include", "hram.h")]
LIB = os.path.join(HERE, "libhram.so")
# the bounds-checked build of the same source (-DHRAM_CHECKED)
LIB_CHECKED = os.path.join(HERE, "libhram_checked.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-ffp-contract=off",
    "-shared",
]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPS)


def _compile(lib: str, extra: list, verbose: bool) -> None:
    tmp = "%s.%d.tmp" % (lib, os.getpid())
    cmd = [nvcc()] + NVCC_FLAGS + extra + ["-I", os.path.join(ROOT, "include"), "-o", tmp] + SRC
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile the library (and its bounds-checked build) if missing or older
    than the sources."""
    if force or stale(LIB):
        _compile(LIB, [], verbose)
    if checked and (force or stale(LIB_CHECKED)):
        _compile(LIB_CHECKED, ["-DHRAM_CHECKED"], verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
