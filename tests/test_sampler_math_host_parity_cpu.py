"""The kernels' sampler building blocks against the oracle's, on the host
(CPU, no GPU).

csrc/sampling.cuh compiles as plain C++ on the host with the same correctly
rounded float operations as on the device; the oracle (oracle/euler_oracle.c)
implements the same written definitions on its own.  This links both into one
test program and compares, bit for bit: the Philox4x32-10 block, the uniform
mapping, exp / log / expm1 / log1p over dense samples of their whole range
(special values included), and Loader's log-pmfs of the binomial and Poisson
laws over the arguments the rejection samplers use.  A drift between the two
sides shows here first; the GPU parity tests check the kernels end to end.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNEL_HEADER = os.path.join(ROOT, "paper_2402_13259_gb300", "csrc", "sampling.cuh")
ORACLE_SRC = os.path.join(ROOT, "oracle", "euler_oracle.c")

ADAPTER = r"""
#include "%s"
/* the oracle's file-local helpers, reachable from the test program */
float t_logpmf_binom(int k, int n, float p, float q) { return logpmf_binom(k, n, p, q); }
float t_logpmf_pois(int k, float lam) { return logpmf_pois(k, lam); }
""" % ORACLE_SRC

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "%s"
#include "%s"
extern "C" float t_logpmf_binom(int k, int n, float p, float q);
extern "C" float t_logpmf_pois(int k, float lam);
using namespace eulernet;
static float f_of(uint32_t b) { float x; std::memcpy(&x, &b, 4); return x; }
static bool same(float a, float b) { return std::memcmp(&a, &b, 4) == 0; }
static long bad = 0, n = 0;
static void check(bool ok, const char* what, float x) {
  ++n;
  if (!ok && bad++ < 8) std::printf("# %%s differs at %%a\n", what, x);
}
int main() {
  // Philox4x32-10 blocks and the uniforms of one stream
  uint32_t s = 12345u;
  for (int t = 0; t < 200000; ++t) {
    s = s * 1664525u + 1013904223u; const uint32_t k0 = s;
    s = s * 1664525u + 1013904223u; const uint32_t k1 = s;
    s = s * 1664525u + 1013904223u; const uint32_t st = s & 0xffffffu;
    s = s * 1664525u + 1013904223u; const uint32_t rep = s;
    const uint32_t purpose = (uint32_t)(t %% 3), station = st, step = (uint32_t)t;
    PhiloxStream ps;
    ps.init(k0, k1, purpose, station, step, rep);
    ps.refill();
    const uint32_t ctr[4] = {purpose << 24, station, step, rep}, key[2] = {k0, k1};
    uint32_t out[4];
    eo_philox4x32_10(ctr, key, out);
    check(ps.w0 == out[0] && ps.w1 == out[1] && ps.w2 == out[2] && ps.w3 == out[3], "philox", 0.0f);
  }
  // exp and expm1: every 61st float of [-104, 89], both signs of zero, infinities, NaN
  for (uint64_t b = 0; b < 0x100000000ull; b += 61) {
    const float x = f_of((uint32_t)b);
    if (!(x > -104.0f && x < 89.0f)) continue;
    check(same(fm::exp(x), eo_expf(x)), "exp", x);
    check(same(fm::expm1(x), eo_expm1f(x)), "expm1", x);
  }
  const float specials[] = {0.0f, -0.0f, INFINITY, -INFINITY, NAN, 88.72283935546875f, -103.97207641601562f,
                            1e-30f, -1e-30f, 0.3465735912322998f, -0.3465735912322998f};
  for (float x : specials) {
    check(same(fm::exp(x), eo_expf(x)), "exp", x);
    check(same(fm::expm1(x), eo_expm1f(x)), "expm1", x);
    check(same(fm::log(x), eo_logf(x)), "log", x);
  }
  // log: every 53rd positive float (subnormals included); log1p: every 53rd float of (-1, 2^40)
  for (uint64_t b = 1; b < 0x7f800000ull; b += 53) {
    const float x = f_of((uint32_t)b);
    check(same(fm::log(x), eo_logf(x)), "log", x);
  }
  for (uint64_t b = 0; b < 0x100000000ull; b += 53) {
    const float x = f_of((uint32_t)b);
    if (!(x > -1.0f && x < 1.0995116e12f)) continue;
    check(same(fm::log1p(x), eo_log1pf(x)), "log1p", x);
  }
  // Loader's log-pmfs over the rejection samplers' arguments
  for (int nn = 20; nn < 200000; nn = nn + 1 + nn / 9)
    for (int pi = 1; pi <= 50; ++pi) {
      const float p = (float)pi / 100.0f, q = 1.0f - p;
      if ((float)nn * p < 10.0f) continue;  // BTRS's domain: n p >= 10, p <= 1/2
      const float se = stirling_err((float)nn);
      for (int k = 0; k <= nn; k += 1 + nn / 97)
        check(same(log_binom_pmf(k, nn, p, q, se), t_logpmf_binom(k, nn, p, q)), "log_binom_pmf", (float)k);
      check(same(log_binom_pmf(nn, nn, p, q, se), t_logpmf_binom(nn, nn, p, q)), "log_binom_pmf", (float)nn);
    }
  for (int li = 0; li < 3000; ++li) {
    const float lam = 10.0f + (float)li * 0.731f;  // PTRS's domain: lambda >= 10
    for (int k = 0; k < (int)(4.0f * lam) + 20; k += 1 + (int)(lam / 40.0f))
      check(same(log_pois_pmf(k, lam), t_logpmf_pois(k, lam)), "log_pois_pmf", (float)k);
  }
  std::printf("%%ld %%ld\n", bad, n);
  return bad != 0;
}
""" % (os.path.join(ROOT, "oracle", "euler_oracle.h"), KERNEL_HEADER)


def test_sampler_building_blocks_match_the_oracle(tmp_path):
    ada = tmp_path / "oracle_adapter.c"
    prog = tmp_path / "parity.cpp"
    exe = tmp_path / "parity"
    ada.write_text(ADAPTER)
    prog.write_text(PROGRAM)
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math"]
    try:
        subprocess.run(["gcc", *flags, "-std=c11", "-c", str(ada), "-o", str(tmp_path / "a.o"),
                        "-I", os.path.join(ROOT, "oracle")], check=True, capture_output=True, text=True)
        subprocess.run(["g++", *flags, "-std=c++17", str(prog), str(tmp_path / "a.o"), "-o", str(exe), "-lm"],
                       check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no host C/C++ compiler")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=900)
    lines = r.stdout.strip().splitlines()
    bad, n = map(int, lines[-1].split())
    assert n > 50_000_000
    assert r.returncode == 0 and bad == 0, "\n".join(lines)
