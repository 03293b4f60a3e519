"""Builds libfit.so in place with nvcc for sm_103a (GB300).

Used by ``__graft_entry__.build()`` and on first import of the binding when the
library is missing or older than its sources.  One translation unit, one
``-gencode``: a few seconds on any host with nvcc, no GPU needed.
"""
from __future__ import annotations

import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libfit.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps() -> list:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def command(out: str = LIB) -> list:
    return [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v", "-I" + INCLUDE,
            "-Xcompiler", "-fPIC", "-shared", *sources(), "-o", out]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run(command(tmp), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed building libfit.so:\n" + r.stdout + r.stderr)
    if verbose:
        print(r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
