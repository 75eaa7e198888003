"""Build libsk.so in-tree with nvcc for sm_103a (no JIT cache, no torch extension),
and libsk_debug.so, the same sources with -DSK_DEBUG: every global load and store of
the kernels checks its address first and reports a failed check through the plan's
error word (the binding loads it when SK_DEBUG_LIBRARY=1)."""

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsk.so")
DEBUG_LIB = os.path.join(HERE, "libsk_debug.so")
SOURCES = ["sk_api.cu", "sk_batch.cu", "sk_server.cu", "sk_noalloc.cu", "sk_selftest.cu",
           "sk_stream.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _build_one(out: str, defines, verbose: bool):
    tag = "debug" if defines else "release"
    bdir = os.path.join(HERE, "_build", tag)
    os.makedirs(bdir, exist_ok=True)
    procs, objs = [], []
    for s in SOURCES:
        o = os.path.join(bdir, s.replace(".cu", ".o"))
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
               "-fPIC,-ffp-contract=off"] + list(defines) + ["-c", os.path.join(CSRC, s), "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
        objs.append(o)
    for p in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, "nvcc")
    subprocess.run([nvcc(), ARCH, "-shared", "-o", out] + objs + ["-lcudart", "-lpthread", "-ldl"],
                   check=True)
    return out


def build(verbose: bool = False, debug: bool = True):
    """libsk.so, and (debug=True) libsk_debug.so beside it."""
    _build_one(LIB, [], verbose)
    if debug:
        _build_one(DEBUG_LIB, ["-DSK_DEBUG"], verbose)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
