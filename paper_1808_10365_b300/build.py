"""Build libsk.so in-tree with nvcc for sm_103a (no JIT cache, no torch extension)."""

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsk.so")
SOURCES = ["sk_api.cu", "sk_batch.cu", "sk_server.cu", "sk_noalloc.cu", "sk_selftest.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def build(verbose: bool = False):
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = []
    for s in SOURCES:
        o = os.path.join(bdir, s.replace(".cu", ".o"))
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
               "-fPIC,-ffp-contract=off", "-c", os.path.join(CSRC, s), "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
        objs.append(o)
    subprocess.run([nvcc(), ARCH, "-shared", "-o", LIB] + objs + ["-lcudart", "-lpthread", "-ldl"],
                   check=True)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
