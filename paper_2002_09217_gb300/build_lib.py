"""Builds ``libpond.so`` (the CUDA product library) in-tree with nvcc for sm_103a.

``python -m paper_2002_09217_gb300.build_lib`` compiles
``csrc/pond.cu`` (host ABI + kernels) into ``paper_2002_09217_gb300/libpond.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "pond.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("pond_kernels.cuh", "pond_step.cuh", "pond_q16.cuh",
                                                      "pond_q27.cuh")] + [os.path.join(ROOT, "include", "pond.h")]
LIB = os.path.join(HERE, "libpond.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpond")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I" + os.path.join(ROOT, "include"), "-o", tmp] + SRC
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
