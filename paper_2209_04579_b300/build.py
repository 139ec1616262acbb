"""Builds the in-tree CUDA library libtqp.so for sm_103a with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtqp.so")
GEN_LIB = os.path.join(HERE, "libtqpgen.so")
GEN_SRC = os.path.join(HERE, "gen", "datagen.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _nvcc(out, src, verbose=False):
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", tmp, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, out)


def build_gen(force: bool = False) -> str:
    deps = [GEN_SRC, os.path.join(HERE, "..", "include", "tqp_datagen.h")]
    if force or not os.path.exists(GEN_LIB) or any(os.path.getmtime(GEN_LIB) < os.path.getmtime(d) for d in deps):
        _nvcc(GEN_LIB, GEN_SRC)
    return GEN_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    build_gen(force)
    srcs = _sources()
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in srcs):
        return LIB
    _nvcc(LIB, os.path.join(CSRC, "tqp.cu"), verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
