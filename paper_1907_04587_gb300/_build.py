"""Builds libnsn.so (the CUDA path) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnsn.so")
SOURCES = [os.path.join(CSRC, "nsn_host.cu"), os.path.join(CSRC, "nsn_collide.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "nsn_kernels.cuh"), os.path.join(CSRC, "nsn_mlp.cuh"), os.path.join(CSRC, "nsn_mlp_tc.cuh"),
                  os.path.join(CSRC, "nsn_internal.h"), os.path.join(CSRC, "nsn_bits.h"), os.path.join(CSRC, "nsn_hostpar.h"),
                  os.path.join(os.path.dirname(HERE), "include", "nsn.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for p in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        cand = os.path.join(p, "bin", "nvcc") if p else ""
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in DEPS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-Xptxas", "-v" if verbose else "-O3", "-o", tmp, *SOURCES, "-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
