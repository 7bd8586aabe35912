"""Build libbpm.so (the CUDA library behind include/bpm.h) for sm_103a, in tree."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRCS = [os.path.join(HERE, "csrc", f) for f in ("bpm.cu", "corrector.cu")]
DEPS = [os.path.join(HERE, "csrc", f) for f in ("bpm.cu", "corrector.cu", "bpm_kernels.cuh", "fft.cuh")] + \
       [os.path.join(ROOT, "include", f) for f in ("bpm.h", "bpm_corrector.h")]
LIB = os.path.join(HERE, "libbpm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/bpm.cu into libbpm.so next to this file (nvcc, sm_103a)."""
    if not force and not needs_build():
        return LIB
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-I", os.path.join(ROOT, "include"), *SRCS, "-o", LIB + ".tmp", "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
