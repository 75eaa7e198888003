"""Build the generator libraries in-tree: libsynth_cpu.so (gcc) and libsynth_gpu.so (nvcc, sm_103a)."""

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _run(cmd):
    subprocess.run(cmd, check=True)


def build_cpu():
    _run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
          "-D_DEFAULT_SOURCE", "-o", os.path.join(HERE, "libsynth_cpu.so"),
          os.path.join(HERE, "synth_cpu.c"), "-lm"])


def build_gpu():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    _run([nvcc, ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
          "-o", os.path.join(HERE, "libsynth_gpu.so"), os.path.join(HERE, "synth_gpu.cu")])


def build():
    build_cpu()
    build_gpu()


if __name__ == "__main__":
    build()
