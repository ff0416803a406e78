// sampling.cuh -- random streams, float32 elementary functions and samplers
// of the Euler step (arXiv 2402.13259), for sm_103a.
//
// Every function evaluates a fixed sequence of correctly rounded IEEE float
// operations (the library is compiled with -fmad=false -prec-div=true
// -prec-sqrt=true -ftz=false; fused multiply-adds appear only where fmaf is
// written), so a replication's integer trajectory is a pure function of
// (seed, replication, step, station).  The definitions:
//   stream   Philox4x32-10, key = (seed lo, seed hi), counter =
//            (purpose << 24 | block, station, step, replication); purpose 0 =
//            external arrivals, 1 = service (departure, then routing edges in
//            CSR order), 2 = the Erlang time of a departure draw with x > m;
//            words consumed in order.
//   uniform  u = (2 (w >> 9) + 1) 2^-24, exact, in [2^-24, 1 - 2^-24].
//   exp/log/expm1/log1p  argument reduction + truncated Taylor/atanh series.
//   Poisson  inversion for lambda < 10, PTRS (Hoermann 1993) otherwise.
//   Binomial symmetric for p > 1/2; inversion for n p < 10, BTRS (Hoermann
//            1993) otherwise, with Loader's (2000) exact log-pmf.
//   Erlang   minus log of products of <= 4 uniforms for shape <= 8,
//            Marsaglia-Tsang (2000) with polar normals otherwise.
#pragma once

#include <cstdint>
#include <cstring>
#include <cmath>

#if defined(__CUDACC__)
#define EN_HD __host__ __device__ __forceinline__
#define EN_D __device__ __forceinline__
#else
#define EN_HD inline
#define EN_D inline
#endif
// Rarely taken sampler paths (rejection samplers for large means, Erlang
// times) are inlined like the rest unless EN_COLD_OUTLINE is defined (one
// out-of-line copy each: smaller code, but calls and more spills).
#if defined(__CUDACC__) && defined(EN_COLD_OUTLINE)
#define EN_COLD static __device__ __noinline__
#else
#define EN_COLD EN_D
#endif
// The Philox block function is inlined at every draw site unless
// EN_PHILOX_OUTLINE is defined (one out-of-line copy: smaller code).
#if defined(__CUDACC__) && defined(EN_PHILOX_OUTLINE)
#define EN_REFILL __device__ __noinline__
#else
#define EN_REFILL EN_D
#endif

// Branch-probability hints (code placement only: the arithmetic is the same).
#if defined(__CUDACC__) || defined(__GNUC__)
#define EN_LIKELY(c) __builtin_expect(!!(c), 1)
#define EN_UNLIKELY(c) __builtin_expect(!!(c), 0)
#else
#define EN_LIKELY(c) (c)
#define EN_UNLIKELY(c) (c)
#endif

namespace eulernet {

// Error bits latched in the handle's device error word.
constexpr unsigned kErrSamplerCap = 1u;
constexpr unsigned kErrOverflow = 2u;
constexpr unsigned kErrStall = 4u;
constexpr int32_t kStateLimit = 1 << 30;

EN_HD float bits_f(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

EN_HD uint32_t f_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

// ---------------------------------------------------------------------------
// Float32 elementary functions.
// ---------------------------------------------------------------------------
namespace fm {

constexpr float kLn2Hi = 0x1.62e400p-1f;  // ln 2 with 9 trailing zero bits
constexpr float kLn2Lo = 0x1.7f7d1cp-20f;  // ln 2 - kLn2Hi
constexpr float kLog2e = 0x1.715476p+0f;
constexpr float kSqrt2 = 0x1.6a09e6p+0f;
constexpr float kLn2Pi = 0x1.d67f1cp+0f;   // ln(2 pi)

EN_HD float inf() { return bits_f(0x7f800000u); }
EN_HD float qnan() { return bits_f(0x7fc00000u); }

// e^x = 2^k e^r, k = floor(x log2e + 1/2), r = x - k ln2 in two parts;
// e^r by its degree-7 Taylor polynomial in Horner form.
EN_HD float exp(float x) {
  if (EN_UNLIKELY(x != x)) return x;
  if (EN_UNLIKELY(x > 88.72283935546875f)) return inf();
  if (EN_UNLIKELY(x < -103.97207641601562f)) return 0.0f;
  const float k = floorf(x * kLog2e + 0.5f);
  float r = fmaf(-k, kLn2Hi, x);
  r = fmaf(-k, kLn2Lo, r);
  float s = (float)(1.0 / 5040.0);
  s = fmaf(s, r, (float)(1.0 / 720.0));
  s = fmaf(s, r, (float)(1.0 / 120.0));
  s = fmaf(s, r, (float)(1.0 / 24.0));
  s = fmaf(s, r, (float)(1.0 / 6.0));
  s = fmaf(s, r, 0.5f);
  s = fmaf(s, r, 1.0f);
  s = fmaf(s, r, 1.0f);
  const int ki = (int)k;
  if (EN_UNLIKELY(ki < -125)) return (s * bits_f((uint32_t)(ki + 227) << 23)) * 0x1p-100f;
  if (EN_UNLIKELY(ki > 127)) return (s * bits_f((uint32_t)(ki + 126) << 23)) * 2.0f;
  return s * bits_f((uint32_t)(ki + 127) << 23);
}

// ln x = e ln2 + ln(1+f), 1+f in [sqrt(1/2), sqrt(2)); with s = f/(2+f),
// ln(1+f) = 2 atanh s = f - s f + 2 s (s^2/3 + s^4/5 + s^6/7 + s^8/9).
EN_HD float log(float x) {
  if (EN_UNLIKELY(x != x)) return x;
  if (EN_UNLIKELY(x < 0.0f)) return qnan();
  if (EN_UNLIKELY(x == 0.0f)) return -inf();
  if (EN_UNLIKELY(x == inf())) return x;
  int bias = 0;
  if (EN_UNLIKELY(x < 0x1p-126f)) {
    x = x * 0x1p25f;
    bias = -25;
  }
  const uint32_t b = f_bits(x);
  int e = (int)(b >> 23) - 127 + bias;
  float m = bits_f((b & 0x007fffffu) | 0x3f800000u);
  if (m > kSqrt2) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float f = m - 1.0f;
  const float s = f / (2.0f + f);
  const float z = s * s;
  float t = (float)(1.0 / 9.0);
  t = fmaf(t, z, (float)(1.0 / 7.0));
  t = fmaf(t, z, (float)(1.0 / 5.0));
  t = fmaf(t, z, (float)(1.0 / 3.0));
  t = t * z;
  const float sf = s * f;
  const float corr = fmaf(2.0f * s, t, -sf);
  const float lm = f + corr;
  const float ef = (float)e;
  const float lo = fmaf(ef, kLn2Lo, lm);
  return fmaf(ef, kLn2Hi, lo);
}

// fm::exp for an argument known to lie in [-87, 0] (the inversion samplers'
// starting probabilities e^{-lambda}, lambda < 10, and (1 - p)^n = e^{n ln(1-p)}
// with n p < 10, p <= 1/2, so n ln(1-p) > -14): the same operations as
// fm::exp, whose special cases cannot occur there.
EN_HD float exp_neg(float x) {
  const float k = floorf(x * kLog2e + 0.5f);
  float r = fmaf(-k, kLn2Hi, x);
  r = fmaf(-k, kLn2Lo, r);
  float s = (float)(1.0 / 5040.0);
  s = fmaf(s, r, (float)(1.0 / 720.0));
  s = fmaf(s, r, (float)(1.0 / 120.0));
  s = fmaf(s, r, (float)(1.0 / 24.0));
  s = fmaf(s, r, (float)(1.0 / 6.0));
  s = fmaf(s, r, 0.5f);
  s = fmaf(s, r, 1.0f);
  s = fmaf(s, r, 1.0f);
  return s * bits_f((uint32_t)((int)k + 127) << 23);
}

// fm::log for an argument known to be a positive normal finite float (every
// sampler call site but log1p's): the same operations as fm::log, whose
// special cases (NaN, negative, zero, infinity, subnormal) cannot occur there.
EN_HD float log_pos(float x) {
  const uint32_t b = f_bits(x);
  int e = (int)(b >> 23) - 127;
  float m = bits_f((b & 0x007fffffu) | 0x3f800000u);
  if (m > kSqrt2) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float f = m - 1.0f;
  const float s = f / (2.0f + f);
  const float z = s * s;
  float t = (float)(1.0 / 9.0);
  t = fmaf(t, z, (float)(1.0 / 7.0));
  t = fmaf(t, z, (float)(1.0 / 5.0));
  t = fmaf(t, z, (float)(1.0 / 3.0));
  t = t * z;
  const float sf = s * f;
  const float corr = fmaf(2.0f * s, t, -sf);
  const float lm = f + corr;
  const float ef = (float)e;
  const float lo = fmaf(ef, kLn2Lo, lm);
  return fmaf(ef, kLn2Hi, lo);
}

// e^x - 1: Taylor to degree 8 below ln2/2 in magnitude, else exp(x) - 1.
EN_HD float expm1(float x) {
  if (fabsf(x) < 0.3465735912322998f) {
    float s = (float)(1.0 / 40320.0);
    s = fmaf(s, x, (float)(1.0 / 5040.0));
    s = fmaf(s, x, (float)(1.0 / 720.0));
    s = fmaf(s, x, (float)(1.0 / 120.0));
    s = fmaf(s, x, (float)(1.0 / 24.0));
    s = fmaf(s, x, (float)(1.0 / 6.0));
    s = fmaf(s, x, 0.5f);
    return fmaf(x * s, x, x);
  }
  return fm::exp(x) - 1.0f;
}

// ln(1+x) = ln(u) * x / (u - 1), u = 1 + x rounded (Goldberg 1991).
EN_HD float log1p(float x) {
  const float u = 1.0f + x;
  if (u == 1.0f) return x;
  return fm::log(u) * (x / (u - 1.0f));
}

// fm::log1p for x in [-1/2, 0) (the binomial constants' ln(1 - pe), pe <= 1/2):
// 1 + x lies in [1/2, 1), so the logarithm's special cases cannot occur.
EN_HD float log1p_half(float x) {
  const float u = 1.0f + x;
  if (u == 1.0f) return x;
  return fm::log_pos(u) * (x / (u - 1.0f));
}

}  // namespace fm

// ---------------------------------------------------------------------------
// Philox4x32-10 stream.
// ---------------------------------------------------------------------------
struct PhiloxStream {
  uint32_t key0, key1;
  // round keys (key0 + r W0 for r < 10, then key1 + r W1) in constant memory
  // (a kernel parameter), or nullptr: then computed while the block is drawn
  const uint32_t* rk;
  uint32_t ctr0, ctr1, ctr2, ctr3;  // ctr0 holds purpose << 24; block is OR-ed in
  uint32_t w0, w1, w2, w3;          // buffered words, consumed w0 first
  uint32_t left;                    // words remaining in the buffer
  uint32_t block;                   // next block index

  // The stream of another purpose at the same (station, step, replication).
  EN_D PhiloxStream sibling(uint32_t purpose) const {
    PhiloxStream s;
    s.init(key0, key1, purpose, ctr1, ctr2, ctr3, rk);
    return s;
  }

  EN_D void init(uint32_t k0, uint32_t k1, uint32_t purpose, uint32_t station, uint32_t step,
                 uint32_t rep, const uint32_t* round_keys = nullptr) {
    key0 = k0;
    key1 = k1;
    rk = round_keys;
    ctr0 = purpose << 24;
    ctr1 = station;
    ctr2 = step;
    ctr3 = rep;
    left = 0;
    block = 0;
  }

  EN_REFILL void refill() {
    uint32_t x0 = ctr0 | block, x1 = ctr1, x2 = ctr2, x3 = ctr3;
    uint32_t k0 = key0, k1 = key1;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
      const unsigned long long m0 = (unsigned long long)0xD2511F53u * x0;  // one wide multiply
      const unsigned long long m1 = (unsigned long long)0xCD9E8D57u * x2;
      const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
      const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
      const uint32_t r0 = rk ? rk[round] : k0;
      const uint32_t r1 = rk ? rk[10 + round] : k1;
      const uint32_t y0 = hi1 ^ x1 ^ r0;
      const uint32_t y2 = hi0 ^ x3 ^ r1;
      x0 = y0;
      x1 = lo1;
      x2 = y2;
      x3 = lo0;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    w0 = x0;
    w1 = x1;
    w2 = x2;
    w3 = x3;
    left = 4;
    ++block;
  }

  EN_D uint32_t next() {
    if (EN_UNLIKELY(left == 0)) refill();
    const uint32_t w = w0;
    w0 = w1;
    w1 = w2;
    w2 = w3;
    --left;
    return w;
  }

  // (w >> 8) | 1 is the odd integer 2 (w >> 9) + 1.
  EN_D float uniform() {
    const uint32_t w = next();
    return (float)((w >> 8) | 1u) * 0x1p-24f;
  }
};

// Per-launch sampler context: reciprocal table 1/k (k < 64) in shared memory,
// rejection cap, latched error bits.
struct SamplerCtx {
  const float* rinv;
  int cap;
  unsigned err;
};

// ---------------------------------------------------------------------------
// Exact log-probabilities (Loader 2000): Stirling error and deviance bd0.
// ---------------------------------------------------------------------------
EN_D float log_small_factorial(int k) {  // k <= 9, k! exact in float
  float f = 1.0f;
  for (int j = 2; j <= k; ++j) f = f * (float)j;
  return fm::log_pos(f);  // f in [1, 9!]
}

EN_D float stirling_err(float k) {
  if (k < 10.0f) {
    float t = (k + 0.5f) * fm::log_pos(k);  // 1 <= k < 10
    t = t - k;
    t = t + 0.5f * fm::kLn2Pi;
    return log_small_factorial((int)k) - t;
  }
  // 1/(12k) - 1/(360k^3) + 1/(1260k^5), nested in r = 1/k (one division)
  const float r = 1.0f / k;
  const float r2 = r * r;
  float s = (float)(1.0 / 1260.0) * r2;
  s = (float)(1.0 / 360.0) - s;
  s = s * r2;
  s = (float)(1.0 / 12.0) - s;
  return s * r;
}

EN_D float deviance(float x, float m) {  // x ln(x/m) + m - x
  if (x == 0.0f) return m;
  const float d = x - m;
  if (fabsf(d) < 0.1f * (x + m)) {
    // odd series in v = d/(x+m), five terms, the term of v^(2j+1) times the
    // float constant 1/(2j+1)
    const float v = d / (x + m);
    float s = d * v;
    float ej = 2.0f * x * v;
    const float v2 = v * v;
    ej = ej * v2;
    s = s + ej * (float)(1.0 / 3.0);
    ej = ej * v2;
    s = s + ej * (float)(1.0 / 5.0);
    ej = ej * v2;
    s = s + ej * (float)(1.0 / 7.0);
    ej = ej * v2;
    s = s + ej * (float)(1.0 / 9.0);
    ej = ej * v2;
    s = s + ej * (float)(1.0 / 11.0);
    return s;
  }
  return x * fm::log_pos(x / m) + m - x;  // x >= 1, m >= 10
}

EN_D float log_pois_pmf(int k, float lam) {
  if (k == 0) return -lam;
  const float kf = (float)k;
  if (k < 10) return kf * fm::log_pos(lam) - lam - log_small_factorial(k);  // lam >= 10
  const float t = fm::kLn2Pi + fm::log_pos(kf);
  float r = -0.5f * t;
  r = r - stirling_err(kf);
  return r - deviance(kf, lam);
}

// se_n: stirling_err((float)n), which depends on n only (a BTRS draw computes
// it once for all its log tests).
EN_D float log_binom_pmf(int k, int n, float p, float q, float se_n) {
  const float nf = (float)n;
  if (k == 0) return nf * fm::log1p_half(-p);  // p in (0, 1/2]
  if (k == n) return nf * fm::log_pos(p);  // n p >= 10, p <= 1/2
  const float kf = (float)k;
  const float rf = (float)(n - k);
  // lc = se_n - d(k) - d(n-k) - bd0(k, np) - bd0(n-k, nq), subtracted in that
  // order, with one inlined copy of each term's code (smaller kernels)
  float lc = se_n;
#pragma unroll 1
  for (int t = 0; t < 2; ++t) lc = lc - stirling_err(t == 0 ? kf : rf);
#pragma unroll 1
  for (int t = 0; t < 2; ++t) lc = lc - deviance(t == 0 ? kf : rf, t == 0 ? nf * p : nf * q);
  const float lf = fm::kLn2Pi + fm::log_pos(kf) + fm::log1p(-(kf / nf));
  return lc - 0.5f * lf;
}

// ---------------------------------------------------------------------------
// Samplers.
// ---------------------------------------------------------------------------
// Hoermann's PTRS for lam >= 10.
EN_COLD int32_t poisson_ptrs(float lam, PhiloxStream& st, SamplerCtx& cx) {
  const float slam = sqrtf(lam);
  const float b = 0.931f + 2.53f * slam;
  const float a = -0.059f + 0.02483f * b;
  const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
  const float vr = 0.9277f - 3.6224f / (b - 2.0f);
  for (int it = 0; it < cx.cap; ++it) {
    const float U = st.uniform() - 0.5f;
    const float V = st.uniform();
    const float us = 0.5f - fabsf(U);
    const float kf = floorf((2.0f * a / us + b) * U + lam + 0.43f);
    if (us >= 0.07f && V <= vr) return (int32_t)kf;
    if (kf < 0.0f || (us < 0.013f && V > us)) continue;
    if (kf > 1.0e9f) continue;
    const int32_t k = (int32_t)kf;
    const float lhs = fm::log_pos(V * inv_alpha / (a / (us * us) + b));
    if (lhs <= log_pois_pmf(k, lam)) return k;
  }
  cx.err |= kErrSamplerCap;
  return (int32_t)floorf(lam);
}

EN_D int32_t poisson(float lam, PhiloxStream& st, SamplerCtx& cx) {
  if (!(lam > 0.0f)) return 0;
  if (EN_LIKELY(lam < 10.0f)) {
    const float u = st.uniform();
    float p = fm::exp_neg(-lam);  // 0 < lam < 10
    float F = p;
    int32_t k = 0;
    while (u > F) {
      if (EN_UNLIKELY(k == 63)) break;
      k = k + 1;
      p = (p * lam) * cx.rinv[k];
      const float Fn = F + p;
      if (EN_UNLIKELY(Fn == F)) break;
      F = Fn;
    }
    return k;
  }
  return poisson_ptrs(lam, st, cx);
}

// Constants of one binomial success probability p, as the sampler uses them:
// c0 = 0 for p <= 0 (or NaN), 2 for p >= 1, otherwise +pe or -pe where
// pe = min(p, 1 - p) and the sign marks the symmetric case p > 1/2;
// q = 1 - pe, r = pe / q and lq = ln(1 - pe) serve the inversion branch.
// For a probability that is fixed per station or per edge they are computed
// once (on the host, with these same functions); per draw otherwise.
struct BinomConst {
  float c0, q, r, lq;
};

EN_HD BinomConst binom_const(float p) {
  BinomConst b;
  if (!(p > 0.0f)) {
    b.c0 = 0.0f;
    b.q = b.r = b.lq = 0.0f;
    return b;
  }
  if (p >= 1.0f) {
    b.c0 = 2.0f;
    b.q = b.r = b.lq = 0.0f;
    return b;
  }
  const bool flip = p > 0.5f;
  const float pe = flip ? 1.0f - p : p;
  b.q = 1.0f - pe;
  b.r = pe / b.q;
  b.lq = fm::log1p_half(-pe);  // pe in (0, 1/2]
  b.c0 = flip ? -pe : pe;
  return b;
}

// Hoermann's BTRS for Bin(n, p), p <= 1/2, n p >= 10.
EN_COLD int32_t binomial_btrs(int32_t n, float p, float q, PhiloxStream& st, SamplerCtx& cx) {
  const float nf = (float)n;
  const float np = nf * p;
  const float spq = sqrtf(np * q);
  const float b = 1.15f + 2.53f * spq;
  const float a = -0.0873f + 0.0248f * b + 0.01f * p;
  const float c = np + 0.5f;
  const float vr = 0.92f - 4.2f / b;
  const float alpha = (2.83f + 5.1f / b) * spq;
  int32_t mode = (int32_t)floorf((nf + 1.0f) * p);
  if (mode > n) mode = n;
  const float se_n = stirling_err(nf);
  // One inlined copy of the log-pmf serves both its uses: the first pass
  // evaluates it at the mode (lpm, before any draw, as if computed up
  // front), every later pass is a rejection iteration that evaluates it at
  // its candidate k when the squeeze does not accept.
  float lpm = 0.0f, lv = 0.0f;
  int32_t kt = mode, k = 0;
  int it = -1;  // -1: the mode's pass; 0 .. cap-1: rejection iterations
  for (;;) {
    if (it >= 0) {
      if (it >= cx.cap) break;
      ++it;
      const float u = st.uniform() - 0.5f;
      const float v = st.uniform();
      const float us = 0.5f - fabsf(u);
      const float kf = floorf((2.0f * a / us + b) * u + c);
      if (kf < 0.0f || kf > nf) continue;
      k = (int32_t)kf;
      if (us >= 0.07f && v <= vr) return k;
      lv = fm::log_pos(v * alpha / (a / (us * us) + b));
      kt = k;
    }
    const float lp = log_binom_pmf(kt, n, p, q, se_n);
    if (it < 0) {
      lpm = lp;
      it = 0;
      continue;
    }
    if (lv <= lp - lpm) return k;
  }
  cx.err |= kErrSamplerCap;
  return (int32_t)floorf(np);
}

// Bin(n, pe) for pe <= 1/2, q = 1 - pe: inversion for n pe < 10 (using r and
// lq), BTRS otherwise.
EN_D int32_t binomial_half(int32_t n, float p, float q, float r, float lq, PhiloxStream& st,
                           SamplerCtx& cx) {
  const float nf = (float)n;
  const float np = nf * p;
  if (EN_LIKELY(np < 10.0f)) {
    float pk = fm::exp_neg(nf * lq);  // n ln(1 - p) > -14 for n p < 10, p <= 1/2
    float F = pk;
    const float u = st.uniform();
    int32_t k = 0;
    while (u > F) {
      if (k == n || EN_UNLIKELY(k == 63)) break;
      pk = ((pk * (float)(n - k)) * r) * cx.rinv[k + 1];
      k = k + 1;
      const float Fn = F + pk;
      if (EN_UNLIKELY(Fn == F)) break;
      F = Fn;
    }
    return k;
  }
  return binomial_btrs(n, p, q, st, cx);
}

// Bin(n, p) from its constants: zero draws if n = 0 or p <= 0 (Appendix A's
// "zero if the first argument is zero"), n if p >= 1, n - Bin(n, 1 - p) for
// p > 1/2.
EN_D int32_t binomial_c(int32_t n, const BinomConst& bc, PhiloxStream& st, SamplerCtx& cx) {
  if (n <= 0 || bc.c0 == 0.0f) return 0;
  if (bc.c0 >= 1.0f) return n;
  const float pe = fabsf(bc.c0);
  const int32_t k = binomial_half(n, pe, bc.q, bc.r, bc.lq, st, cx);
  return bc.c0 < 0.0f ? n - k : k;
}

EN_D int32_t binomial(int32_t n, float p, PhiloxStream& st, SamplerCtx& cx) {
  return binomial_c(n, binom_const(p), st, cx);
}

EN_D float std_normal(PhiloxStream& st, SamplerCtx& cx) {
  for (int it = 0; it < cx.cap; ++it) {
    const float v1 = 2.0f * st.uniform() - 1.0f;
    const float v2 = 2.0f * st.uniform() - 1.0f;
    const float s = v1 * v1 + v2 * v2;
    if (s < 1.0f) {
      const float t = (-2.0f * fm::log_pos(s)) / s;  // s in [2^-46, 1)
      return v1 * sqrtf(t);
    }
  }
  cx.err |= kErrSamplerCap;
  return 0.0f;
}

EN_COLD float erlang(int32_t k, float rate, PhiloxStream& st, SamplerCtx& cx) {
  if (k <= 0) return 0.0f;
  if (k <= 8) {
    float S = 0.0f;
    int32_t rem = k;
    while (rem > 0) {
      const int32_t g = rem < 4 ? rem : 4;
      float prod = st.uniform();
      for (int32_t j = 1; j < g; ++j) prod = prod * st.uniform();
      S = S - fm::log_pos(prod);  // prod in [2^-96, 1)
      rem = rem - g;
    }
    return S / rate;
  }
  const float d = (float)k - (float)(1.0 / 3.0);
  const float cc = 1.0f / sqrtf(9.0f * d);
  for (int it = 0; it < cx.cap; ++it) {
    const float x = std_normal(st, cx);
    float v = 1.0f + cc * x;
    if (v <= 0.0f) continue;
    v = v * v * v;
    const float u = st.uniform();
    const float x2 = x * x;
    if (u < 1.0f - 0.0331f * (x2 * x2)) return d * v / rate;
    float lu = 0.0f, lv = 0.0f;  // ln u, ln v from one inlined copy of the logarithm
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      const float l = fm::log_pos(t == 0 ? u : v);  // u >= 2^-24; v in [2^-72, 2^78]
      if (t == 0) lu = l;
      else lv = l;
    }
    if (lu < 0.5f * x2 + d * ((1.0f - v) + lv)) return d * v / rate;
  }
  cx.err |= kErrSamplerCap;
  return (float)k / rate;
}

// GenerateDeparture(x, m, mu, h), Lemma 1 / Algorithm 1, split at its last
// draw: this part takes the branch (drawing T ~ Erlang(x - m, m mu) when
// x > m) and returns the binomial that completes D = base + Bin(n, p):
//   x <= m        : Bin(x, p0),                       p0 = 1 - e^{-mu h}
//   x > m, T > h  : Bin(x - m - 1, h / T)
//   x > m, T <= h : (x - m) + Bin(m, 1 - e^{-mu (h - T)})
// T comes from the unit's Erlang stream (purpose 2), the binomial from the
// service stream; callers draw that binomial next, so the draws are exactly
// Algorithm 1's, and lanes on either branch meet again at one binomial.
// With its own stream the Erlang time's groups of four uniforms are whole
// Philox blocks, so the lanes that draw one compute each block together.
struct BinomialArgs {
  int32_t n;
  BinomConst c;
  int32_t base;
  int32_t branch;  // 0: x <= m, 1: T > h, 2: T <= h
  float T;         // the Erlang time (branches 1 and 2)
  float p;         // the binomial's p in branch 2
};

// p0c: the constants of p0 = 1 - e^{-mu h} of this station (fixed per call).
EN_D BinomialArgs departure_branch(int32_t x, int32_t m, float mu, float h, const BinomConst& p0c,
                                   PhiloxStream& st, SamplerCtx& cx) {
  BinomialArgs b;
  b.base = 0;
  b.branch = 0;
  b.T = 0.0f;
  b.p = 0.0f;
  if (EN_LIKELY(x <= m)) {
    b.n = x;
    b.c = p0c;
    return b;
  }
  const float rate = (float)m * mu;
  PhiloxStream es = st.sibling(2u);
  es.refill();  // every Erlang draw takes at least one word
  const float T = erlang(x - m, rate, es, cx);
  b.T = T;
  float pb;
  if (T > h) {
    b.n = x - m - 1;
    pb = h / T;
    b.branch = 1;
  } else {
    b.n = m;
    b.p = -fm::expm1(-(mu * (h - T)));
    pb = b.p;
    b.base = x - m;
    b.branch = 2;
  }
  b.c = binom_const(pb);  // one copy for both branches
  return b;
}

}  // namespace eulernet
