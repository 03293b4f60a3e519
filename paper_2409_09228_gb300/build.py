"""Builds libfit.so in place with nvcc for sm_103a (GB300).

Used by ``__graft_entry__.build()`` and on first import of the binding when the
library is missing or older than its sources.  Every translation unit is
compiled to an object in parallel (one ``-gencode``), then linked: no GPU
needed.
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


FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v", "-Xcompiler", "-fPIC"]


def command(out: str = LIB) -> list:
    """One nvcc command for the whole library (serial over the sources)."""
    return [nvcc(), *FLAGS, "-I" + INCLUDE, "-shared", *sources(), "-o", out]


def compile_commands(objdir: str) -> list:
    """(source, object, command) for every translation unit."""
    out = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        out.append((src, obj, [nvcc(), *FLAGS, "-I" + INCLUDE, "-c", src, "-o", obj]))
    return out


def link_command(objs: list, out: str) -> list:
    return [nvcc(), ARCH, "-shared", *objs, "-o", out]


def build_objects(out: str, verbose: bool = False) -> None:
    """Compiles the sources in parallel and links them into `out`."""
    import shutil
    import tempfile
    objdir = tempfile.mkdtemp(prefix="libfit_obj_")
    try:
        jobs = [(src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True))
                for src, obj, cmd in compile_commands(objdir)]
        failed, logs = [], []
        for src, obj, proc in jobs:
            text, _ = proc.communicate()
            logs.append(text)
            if proc.returncode != 0:
                failed.append(f"{os.path.basename(src)}:\n{text}")
        if failed:
            raise RuntimeError("nvcc failed building libfit.so:\n" + "\n".join(failed))
        r = subprocess.run(link_command([o for _, o, _ in jobs], out), capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed linking libfit.so:\n" + r.stdout + r.stderr)
        if verbose:
            print("".join(logs))
    finally:
        shutil.rmtree(objdir, ignore_errors=True)


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    build_objects(tmp, verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
