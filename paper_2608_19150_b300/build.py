"""Build libbgk_b300.so in-tree for sm_103a (nvcc for the kernels, g++ for host set-up)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbgk_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["bgk_lib.cu", "bgk_batch.cuh", "bgk_mlp.cuh", "bgk_guess.cuh", "bgk_static.cu", "bgk_probe.cu", "bgk_host.cpp", "bgk_kernels.cuh", "bgk_internal.h", "bgk_tables.h"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(INC, "bgk.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    host_o = os.path.join(BUILD, "bgk_host.o")
    # host set-up: no contraction, the face signs must match the device bit for bit
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                           "-I", INC, "-c", os.path.join(CSRC, "bgk_host.cpp"), "-o", host_o])
    cmd = [NVCC] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                           "-shared", "-I", INC, os.path.join(CSRC, "bgk_lib.cu"),
                           os.path.join(CSRC, "bgk_static.cu"), os.path.join(CSRC, "bgk_probe.cu"), host_o, "-o", LIB + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
