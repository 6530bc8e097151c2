"""Builds the CUDA library libampcg.so in-tree for sm_103a with nvcc.

Every csrc/*.cu is one translation unit: the host side of the C ABI
(ampcg.cu) and the units that hold the persistent kernels' instantiations
(loop_*.cu, batched_kernels.cu).  They compile in parallel to objects, which
are then linked into the shared library.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libampcg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ampcg.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC"]


def units() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def sources() -> list[str]:
    return units() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources() + [HEADER])


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile csrc/*.cu (in parallel) and link _build/libampcg.so."""
    if not force and not stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = f".{os.getpid()}"

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
        return obj

    jobs = jobs or min(len(units()), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, units()))
    tmp = LIB + tag + ".tmp"
    try:
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
