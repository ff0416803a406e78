"""Build the in-tree CUDA library ``libeulernet.so`` (sm_103a only).

The translation units are compiled in parallel with nvcc and linked
against the shared CUDA runtime.  Float semantics: no multiply-add
contraction, IEEE division and square root, denormals kept -- the samplers
rely on every float operation being the correctly rounded one written in the
source.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeulernet.so")
SOURCES = ["kernels.cu", "pipeline.cu", "abi.cu", "noalloc.cu", "batch.cu", "sojourn.cu", "coupled.cu"]
HEADERS = ["sampling.cuh", "internal.h", "handle.h", "unit.cuh", "tile.cuh", "hbm_step.cuh", os.path.join("..", "..", "include", "eulernet.h")]

NVCC = os.environ.get("NVCC", "nvcc")
# extra nvcc arguments for tuning builds (e.g. "-DEN_HBM_MIN_BLOCKS=3"); the
# objects are not rebuilt when only this changes, so pass --force with it
EXTRA_FLAGS = os.environ.get("EULERNET_NVCC_EXTRA", "").split()
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
    "-ftz=false", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off,-fno-fast-math,-fvisibility=hidden", "-Xptxas",
    "-warn-spills",
]


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.normpath(os.path.join(CSRC, h)) for h in HEADERS]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer(o, [s] + headers):
            extra = ["-Xptxas", "-v"] if verbose else []
            jobs.append([NVCC, *FLAGS, *EXTRA_FLAGS, *extra, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if force or jobs or _newer(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, *ARCH, "-shared", "--cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
