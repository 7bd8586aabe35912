"""Build libbpm.so (the CUDA library behind include/bpm.h) for sm_103a, in tree."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# translation units: the host side and C ABI (bpm.cu), the kernels of each
# group of transform lengths (ops_*.cu), the batched kernel, the corrector;
# the slowest first, so that the parallel compilation ends sooner
SRCS = [os.path.join(HERE, "csrc", f) for f in
        ("ops_1024.cu", "ops_2048.cu", "batch0.cu", "batch1.cu", "batch2.cu", "ops_512.cu", "ops_256.cu",
         "ops_384.cu", "ops_small.cu", "bpm.cu", "corrector.cu")]
DEPS = SRCS + [os.path.join(HERE, "csrc", f) for f in
               ("bpm_kernels.cuh", "bpm_args.cuh", "bpm_aux_kernels.cuh", "bpm_ops.cuh", "bpm_ops.h", "batch.cuh",
                "fft.cuh")] + \
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
    # the translation units compile in parallel (one nvcc each, identical
    # flags), then link; split compilation inside a unit (--split-compile)
    # was measured to slow the batched kernel by 13 % and is not used
    common = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs = [LIB + "." + os.path.splitext(os.path.basename(src))[0] + ".o" for src in SRCS]
    procs = [subprocess.Popen([*common, "-c", src, "-o", obj]) for src, obj in zip(SRCS, objs)]
    codes = [pr.wait() for pr in procs]
    if any(codes):
        raise subprocess.CalledProcessError(max(codes), "nvcc")
    subprocess.run([NVCC, *ARCH, "-shared", *objs, "-o", LIB + ".tmp", "-lcudart"], check=True)
    for obj in objs:
        os.remove(obj)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
