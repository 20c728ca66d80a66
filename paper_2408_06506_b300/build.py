"""Build libtacsl.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2408_06506_b300.build [--force]

The library is one translation unit (csrc/tacsl.cu includes the kernel headers), so
the build is a single nvcc call; it is skipped when the .so is newer than every
source and header.
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
LIB = os.path.join(PKG, "libtacsl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def nvcc_command(out: str, extra=()) -> list:
    return (["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
             "-I", INCLUDE, "-o", out, os.path.join(CSRC, "tacsl.cu")] + list(extra))


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = nvcc_command(tmp, ["-Xptxas", "-v"] if verbose else [])
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
