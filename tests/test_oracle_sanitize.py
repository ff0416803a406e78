"""The CPU oracle and the exact DES under AddressSanitizer and
UndefinedBehaviorSanitizer: a C driver (oracle_sanitize_main.c) calls every
entry point on networks that reach every sampler branch; any out-of-bounds
access, use after free, leak or undefined arithmetic fails the run."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_and_des_are_clean_under_sanitizers():
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    tmp = tempfile.mkdtemp(prefix="oracle_san_")
    try:
        exe = os.path.join(tmp, "san")
        cmd = ["gcc", "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
               "-ffp-contract=off", "-fno-fast-math", "-I", os.path.join(ROOT, "oracle"), "-o", exe,
               os.path.join(ROOT, "tests", "oracle_sanitize_main.c"),
               os.path.join(ROOT, "oracle", "euler_oracle.c"), os.path.join(ROOT, "oracle", "exact_des.c"),
               "-lm"]
        b = subprocess.run(cmd, capture_output=True, text=True)
        if b.returncode != 0 and "sanitize" in b.stderr:
            pytest.skip("gcc without sanitizer runtimes: " + b.stderr[-200:])
        assert b.returncode == 0, b.stderr[-2000:]
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
                   UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
        assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout[-1000:], r.stderr[-3000:])
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
