"""The kernels' check-free elementary functions equal the general ones on
their stated domains (CPU, no GPU).

csrc/sampling.cuh compiles as plain C++ on the host, where its float
operations are the same correctly rounded IEEE operations as on the device
(no contraction, fma only where written).  fm::log_pos, fm::exp_neg and
fm::log1p_half drop special-case tests that cannot fire at their call sites;
this checks, over a dense sample of every binade of each domain and its end
points, that they return the same bits as fm::log, fm::exp and fm::log1p.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2402_13259_gb300", "csrc", "sampling.cuh")

SRC = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "%s"
using namespace eulernet;
static float f_of(uint32_t b) { float x; std::memcpy(&x, &b, 4); return x; }
static uint32_t b_of(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }
int main() {
  long bad = 0, n = 0;
  // log_pos: every positive normal finite float, stride 97 through the bit patterns
  for (uint64_t b = 0x00800000u; b < 0x7f800000u; b += 97) {
    const float x = f_of((uint32_t)b);
    ++n; bad += b_of(fm::log(x)) != b_of(fm::log_pos(x));
  }
  bad += b_of(fm::log(f_of(0x7f7fffffu))) != b_of(fm::log_pos(f_of(0x7f7fffffu)));
  // exp_neg: [-87, 0], every 7th float, and both ends
  for (uint64_t b = 0x80000000u; f_of((uint32_t)b) >= -87.0f; b += 7) {
    const float x = f_of((uint32_t)b);
    ++n; bad += b_of(fm::exp(x)) != b_of(fm::exp_neg(x));
  }
  bad += b_of(fm::exp(-87.0f)) != b_of(fm::exp_neg(-87.0f));
  // log1p_half: [-1/2, 0), every 5th float, and -1/2
  for (uint64_t b = 0x80000001u; f_of((uint32_t)b) >= -0.5f; b += 5) {
    const float x = f_of((uint32_t)b);
    ++n; bad += b_of(fm::log1p(x)) != b_of(fm::log1p_half(x));
  }
  bad += b_of(fm::log1p(-0.5f)) != b_of(fm::log1p_half(-0.5f));
  std::printf("%%ld %%ld\n", bad, n);
  return bad != 0;
}
""" % HEADER


def test_check_free_functions_match_on_their_domains(tmp_path):
    src = tmp_path / "fastpaths.cpp"
    exe = tmp_path / "fastpaths"
    src.write_text(SRC)
    try:
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", str(src), "-o",
                        str(exe), "-lm"], check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no host C++ compiler")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    bad, n = map(int, r.stdout.split())
    assert n > 20_000_000
    assert r.returncode == 0 and bad == 0, f"{bad} of {n} arguments differ"
