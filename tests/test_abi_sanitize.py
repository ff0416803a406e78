"""The C ABI's host code under AddressSanitizer and UndefinedBehaviorSanitizer:
the library is rebuilt with the host compiler's sanitizers and loaded into a
Python process that preloads their runtimes; euler_net_create runs its whole
host side (validation, levels, split probabilities, reverse graph, arrival
columns) on valid networks of both arrival kinds and on each kind of invalid
one.  Without a GPU the valid ones end at the first CUDA call with
EULER_ERR_CUDA and free what they built, which the sanitizers check too."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_13259_gb300", "csrc")
SOURCES = ["kernels.cu", "pipeline.cu", "abi.cu", "noalloc.cu", "batch.cu", "sojourn.cu", "coupled.cu"]

DRIVER = r'''
import ctypes as C, sys
import numpy as np
L = C.CDLL(sys.argv[1])
vp, i32 = C.c_void_p, C.c_int32
class Arr(C.Structure):
    _fields_ = [("kind", i32), ("w", vp), ("a", C.c_double), ("b", C.c_double), ("period", C.c_double),
                ("phase", C.c_double), ("table", vp), ("table_len", i32), ("tab_dt", C.c_double)]
L.euler_net_create.argtypes = [C.POINTER(vp), i32, vp, vp, vp, vp, vp, C.POINTER(Arr), vp]
L.euler_stats_len.restype = C.c_int64
L.euler_stats_len.argtypes = [i32, C.c_int64]
L.euler_num_steps.restype = C.c_int64
L.euler_num_steps.argtypes = [C.c_double, C.c_double]
def create(n, edges, kind=1, N0=None):
    rows = [[] for _ in range(n)]
    for a, b, p in edges:
        rows[a].append((b, p))
    rp = np.zeros(n + 1, np.int32); col = []; prob = []
    for i in range(n):
        rp[i + 1] = rp[i] + len(rows[i]); col += [b for b, _ in rows[i]]; prob += [p for _, p in rows[i]]
    col = np.array(col or [0], np.int32); prob = np.array(prob or [0.0])
    sv = np.full(n, 2, np.int32); mu = np.ones(n)
    w = np.arange(1, n + 1, dtype=float); tab = np.ones(3 * n)
    arr = Arr(kind, w.ctypes.data, 1.0, 0.3, 5.0, 0.1, tab.ctypes.data, 3, 0.5)
    n0 = None if N0 is None else np.array(N0, np.int32)
    h = vp()
    return L.euler_net_create(C.byref(h), n, rp.ctypes.data, col.ctypes.data, prob.ctypes.data,
                              sv.ctypes.data, mu.ctypes.data, C.byref(arr),
                              None if n0 is None else n0.ctypes.data)
dag = [(0, 1, 0.5), (0, 2, 0.5), (1, 3, 1.0), (2, 4, 0.3), (3, 4, 0.9)]
codes = [create(5, dag, 1, [1, 2, 3, 4, 5]), create(5, dag, 2), create(1, [], 0),
         create(3, [(0, 1, 0.5), (1, 2, 0.5), (2, 0, 0.5)]), create(2, [(0, 1, 1.5)]),
         create(2, [(0, 0, 0.5)]), create(4, [(0, 5, 0.5)])]
assert L.euler_stats_len(5, 7) == 58 and L.euler_num_steps(0.01, 1.0) == 100
print(codes)
'''


def test_abi_host_code_is_clean_under_sanitizers():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the valid networks would reach the device")
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None or shutil.which("gcc") is None:
        pytest.skip("no nvcc or gcc")
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["gcc", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("no sanitizer runtimes")
    tmp = tempfile.mkdtemp(prefix="abi_san_")
    try:
        flags = ["-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "-fmad=false",
                 "-prec-div=true", "-prec-sqrt=true", "-ftz=false", "-Xcompiler",
                 "-fPIC,-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer,-ffp-contract=off"]

        def compile_one(src):
            obj = os.path.join(tmp, src.replace(".cu", ".o"))
            r = subprocess.run([nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj],
                               capture_output=True, text=True)
            return obj, r

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            results = list(ex.map(compile_one, SOURCES))
        for obj, r in results:
            assert r.returncode == 0, r.stderr[-2000:]
        lib = os.path.join(tmp, "libeulernet_san.so")
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "--cudart", "shared",
                            "-Xcompiler", "-fsanitize=address,-fsanitize=undefined", "-o", lib,
                            *[o for o, _ in results]], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}",
                   ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
        run = subprocess.run([sys.executable, "-c", DRIVER, lib], capture_output=True, text=True,
                             timeout=600, env=env)
        assert run.returncode == 0, (run.stdout[-1000:], run.stderr[-3000:])
        # EULER_ERR_CUDA for the valid networks (no device), argument and cycle errors otherwise
        assert run.stdout.strip() == "[-3, -3, -3, -2, -1, -2, -1]", run.stdout
        assert "ERROR: AddressSanitizer" not in run.stderr and "runtime error" not in run.stderr, run.stderr[-3000:]
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
