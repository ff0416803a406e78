"""The kernels' samplers against the oracle's, draw for draw, on the host
(CPU, no GPU).

csrc/sampling.cuh compiles as plain C++ on the host with the same correctly
rounded float operations as on the device.  With every stream keyed as the
oracle's eo_draw_* functions key theirs (seed, purpose 1, station 0, step 0,
replication j), the kernels' Poisson, binomial, Erlang, normal and
departure (Algorithm 1) samplers must return exactly the oracle's draws, over
parameters that reach every branch: inversion and the PTRS / BTRS rejection
samplers, the binomial's symmetric and degenerate cases, the small-shape and
Marsaglia-Tsang Erlang samplers, and both branches of Algorithm 1's x > m
case.  The GPU parity tests check the kernels themselves end to end.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNEL_HEADER = os.path.join(ROOT, "paper_2402_13259_gb300", "csrc", "sampling.cuh")
ORACLE_DIR = os.path.join(ROOT, "oracle")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include "%s"
#include "%s"
using namespace eulernet;
static const uint64_t kSeed = 0x5eed1234abcdull;
static const int kCount = 4000;
static float rinv[64];
static long bad = 0, n = 0;
static PhiloxStream stream_of(int64_t j) {
  PhiloxStream s;
  s.init((uint32_t)kSeed, (uint32_t)(kSeed >> 32), 1u, 0u, 0u, (uint32_t)j);
  return s;
}
static void report(bool ok, const char* what, double a, double b) {
  ++n;
  if (!ok && bad++ < 8) std::printf("# %%s: %%g %%g\n", what, a, b);
}
int main() {
  rinv[0] = 0.0f;
  for (int k = 1; k < 64; ++k) rinv[k] = 1.0f / (float)k;
  SamplerCtx cx{rinv, 1000, 0u};
  std::vector<int32_t> oi(kCount);
  std::vector<float> of(kCount);
  const float lams[] = {0.0f, 1e-3f, 0.3f, 2.0f, 9.99f, 10.0f, 10.5f, 37.0f, 1000.0f, 123456.7f};
  for (float lam : lams) {
    eo_draw_poisson(lam, kSeed, kCount, oi.data());
    for (int j = 0; j < kCount; ++j) {
      PhiloxStream s = stream_of(j);
      const int32_t k = poisson(lam, s, cx);
      report(k == oi[j], "poisson", lam, k);
    }
  }
  const int32_t ns[] = {0, 1, 7, 20, 21, 100, 999, 5000, 123457};
  const float ps[] = {0.0f, 1e-4f, 0.01f, 0.0999f, 0.1f, 0.3f, 0.5f, 0.51f, 0.9f, 0.999f, 1.0f};
  for (int32_t nn : ns)
    for (float p : ps) {
      eo_draw_binomial(nn, p, kSeed, kCount, oi.data());
      const BinomConst bc = binom_const(p);
      for (int j = 0; j < kCount; ++j) {
        PhiloxStream s = stream_of(j);
        const int32_t k = binomial_c(nn, bc, s, cx);
        report(k == oi[j], "binomial", nn * 1000.0 + p, k);
      }
    }
  const int32_t ks[] = {0, 1, 2, 3, 4, 5, 8, 9, 20, 500};
  for (int32_t k : ks) {
    eo_draw_gamma(k, 3.7f, kSeed, kCount, of.data());
    for (int j = 0; j < kCount; ++j) {
      PhiloxStream s = stream_of(j);
      const float g = erlang(k, 3.7f, s, cx);
      report(std::memcmp(&g, &of[j], 4) == 0, "erlang", k, g);
    }
  }
  eo_draw_normal(kSeed, kCount, of.data());
  for (int j = 0; j < kCount; ++j) {
    PhiloxStream s = stream_of(j);
    const float z = std_normal(s, cx);
    report(std::memcmp(&z, &of[j], 4) == 0, "normal", j, z);
  }
  // Algorithm 1: x <= m, and x > m with T > h and T <= h
  struct Dep { int32_t x, m; double mu, h; };
  const Dep deps[] = {{0, 5, 1.0, 0.01},     {40, 50, 1.0, 0.01},   {50, 50, 2.0, 0.1},
                      {51, 50, 1.0, 0.01},   {60, 50, 1.0, 0.01},   {58, 50, 30.0, 0.1},
                      {700, 100, 1.3, 0.01}, {3000, 1000, 2.0, 0.05}, {12, 3, 9.0, 0.2},
                      {900, 800, 0.5, 0.01}, {20000, 15000, 1.7, 0.01}};
  for (const Dep& d : deps) {
    eo_draw_departure(d.x, d.m, d.mu, d.h, kSeed, kCount, oi.data());
    const float mu = (float)d.mu, h = (float)d.h;
    const BinomConst p0c = binom_const(-fm::expm1(-(float)(d.mu * d.h)));
    for (int j = 0; j < kCount; ++j) {
      PhiloxStream s = stream_of(j);
      s.refill();
      const BinomialArgs b = departure_branch(d.x, d.m, mu, h, p0c, s, cx);
      const int32_t D = b.base + binomial_c(b.n, b.c, s, cx);
      report(D == oi[j], "departure", d.x * 1e5 + d.m, D);
    }
  }
  std::printf("%%ld %%ld %%u\n", bad, n, cx.err);
  return bad != 0;
}
""" % (os.path.join(ORACLE_DIR, "euler_oracle.h"), KERNEL_HEADER)


def test_samplers_draw_what_the_oracle_draws(tmp_path):
    from oracle import oracle as O
    so = O.build_oracle()
    prog = tmp_path / "draws.cpp"
    exe = tmp_path / "draws"
    prog.write_text(PROGRAM)
    try:
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", str(prog), "-o", str(exe),
                        so, "-Wl,-rpath," + os.path.dirname(so), "-lm"], check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no host C++ compiler")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    lines = r.stdout.strip().splitlines()
    bad, n, err = map(int, lines[-1].split())
    assert n > 500_000
    assert r.returncode == 0 and bad == 0, "\n".join(lines)
