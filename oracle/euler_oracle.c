/*
 * euler_oracle.c -- TEST INFRASTRUCTURE ONLY (see euler_oracle.h).
 *
 * A deliberately plain, single-threaded, obviously-ordered implementation of
 * the Euler schemes of arXiv 2402.13259.  Every random variate is drawn from a
 * counter-based Philox4x32-10 stream so that the CUDA path, which implements
 * the same written definitions on its own, reproduces every integer exactly.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (contraction off: every float expression below is evaluated with one IEEE
 * rounding per written operation; fused multiply-adds appear only where
 * fmaf() is written explicitly).
 */
#include "euler_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Work counters                                                            */
/* ------------------------------------------------------------------------ */
static int64_t g_cnt[EOC_COUNT];
#define CNT(k) (g_cnt[(k)]++)
void eo_counters_reset(void) { memset(g_cnt, 0, sizeof g_cnt); }
void eo_counters_get(int64_t out[EOC_COUNT]) { memcpy(out, g_cnt, sizeof g_cnt); }

static int32_t g_cap = 1000;  /* rejection-loop iteration cap */
int32_t eo_set_cap(int32_t cap) { int32_t o = g_cap; g_cap = cap > 0 ? cap : 1; return o; }

static int32_t g_grad_center = 0;  /* eo_grad: 1 = centred estimator */
int32_t eo_set_grad_center(int32_t on) { int32_t o = g_grad_center; g_grad_center = on ? 1 : 0; return o; }

static int32_t g_dep_mode = 0;  /* 0 exact, 1 Eq. (1), 2 Eq. (2) */
/* external arrival means of steps lo..hi multiplied by factor (a perturbation
   of the arrival-rate profile for the coupled gradient; off by default) */
static int64_t g_win_lo = 1, g_win_hi = 0;
static double g_win_factor = 1.0;
void eo_set_arrival_window(int64_t lo, int64_t hi, double factor) {
  g_win_lo = lo;
  g_win_hi = hi;
  g_win_factor = factor;
}
int32_t eo_set_departure_mode(int32_t mode) {
  int32_t o = g_dep_mode;
  g_dep_mode = (mode >= 0 && mode <= 2) ? mode : 0;
  return o;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random      */
/* numbers: as easy as 1, 2, 3").  Ten rounds; the key is bumped by the     */
/* Weyl constants between rounds.                                           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void eo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One random stream: key = (seed lo, seed hi); counter = (purpose<<24 | block,
 * station, step, replication).  Words are consumed in order x, y, z, w of
 * block 0, then block 1, ... */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t buf[4];
  int used;      /* words of buf already consumed (4 = need a new block) */
  uint32_t blk;  /* next block index                                       */
} stream_t;

static void stream_init(stream_t* s, uint64_t seed, uint32_t purpose, uint32_t station,
                        uint32_t step, uint32_t rep) {
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->ctr[0] = purpose << 24;
  s->ctr[1] = station;
  s->ctr[2] = step;
  s->ctr[3] = rep;
  s->used = 4;
  s->blk = 0;
}

/* The stream of another purpose at the same (station, step, replication). */
static void stream_sibling(stream_t* s, const stream_t* of, uint32_t purpose) {
  *s = *of;
  s->ctr[0] = purpose << 24;
  s->used = 4;
  s->blk = 0;
}

static uint32_t next_word(stream_t* s) {
  if (s->used == 4) {
    uint32_t c[4] = {s->ctr[0] | s->blk, s->ctr[1], s->ctr[2], s->ctr[3]};
    eo_philox4x32_10(c, s->key, s->buf);
    s->blk++;
    s->used = 0;
    CNT(EOC_PHILOX_BLOCKS);
  }
  return s->buf[s->used++];
}

/* Uniform on the odd multiples of 2^-24: u = (2*(w>>9)+1) * 2^-24, which lies
 * in [2^-24, 1-2^-24], is exact in float32, and is symmetric about 1/2. */
static float next_uniform(stream_t* s) {
  uint32_t w = next_word(s);
  uint32_t odd = ((w >> 9) << 1) | 1u;
  CNT(EOC_UNIFORMS);
  return (float)odd * 5.9604644775390625e-8f; /* 2^-24 */
}

/* ------------------------------------------------------------------------ */
/* Float32 elementary functions, written from their mathematical            */
/* definitions (argument reduction + truncated series), so that both sides */
/* of the parity check evaluate exactly the same sequence of IEEE           */
/* operations.  No libm float function is called.                          */
/* ------------------------------------------------------------------------ */
static inline float bits_to_f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static inline uint32_t f_to_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

#define LN2_HI 0x1.62e400p-1f      /* ln 2 with the low 9 mantissa bits zero  */
#define LN2_LO 0x1.7f7d1cp-20f     /* ln 2 - LN2_HI, rounded                  */
#define LOG2E  0x1.715476p+0f      /* 1/ln 2                                  */
#define SQRT2F 0x1.6a09e6p+0f
#define LN_2PI 0x1.d67f1cp+0f      /* ln(2*pi) = 1.83787706...                */

/* exp(x): x = k ln2 + r with k = floor(x log2e + 1/2), r by a two-constant
 * reduction; e^r from its Taylor series to degree 7 (|r| <= ~0.35, the
 * dropped term is below 0.1 ulp); scaled by 2^k through the exponent field. */
float eo_expf(float x) {
  if (x != x) return x;
  if (x > 88.72283935546875f) return INFINITY;
  if (x < -103.97207641601562f) return 0.0f;
  float kf = floorf(x * LOG2E + 0.5f);
  float r = fmaf(-kf, LN2_HI, x);
  r = fmaf(-kf, LN2_LO, r);
  float p = (float)(1.0 / 5040.0);
  p = fmaf(p, r, (float)(1.0 / 720.0));
  p = fmaf(p, r, (float)(1.0 / 120.0));
  p = fmaf(p, r, (float)(1.0 / 24.0));
  p = fmaf(p, r, (float)(1.0 / 6.0));
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  int k = (int)kf;
  if (k < -125) return (p * bits_to_f((uint32_t)(k + 100 + 127) << 23)) * 0x1p-100f;
  if (k > 127) return (p * bits_to_f((uint32_t)(k - 1 + 127) << 23)) * 2.0f;
  return p * bits_to_f((uint32_t)(k + 127) << 23);
}

/* log(x) for x > 0: x = 2^e * m with m in [sqrt(1/2), sqrt(2)); with f = m-1
 * and s = f/(2+f), log(1+f) = 2 atanh(s) = f - s*f + 2s*(s^2/3 + s^4/5 +
 * s^6/7 + s^8/9) (|s| <= 0.172, dropped terms below 1e-9 relative). */
float eo_logf(float x) {
  if (x != x) return x;
  if (x < 0.0f) return NAN;
  if (x == 0.0f) return -INFINITY;
  if (x == INFINITY) return x;
  int eadj = 0;
  if (x < 0x1p-126f) { x = x * 0x1p25f; eadj = -25; }
  uint32_t b = f_to_bits(x);
  int e = (int)(b >> 23) - 127 + eadj;
  float m = bits_to_f((b & 0x007fffffu) | 0x3f800000u);
  if (m > SQRT2F) { m = m * 0.5f; e = e + 1; }
  float f = m - 1.0f;
  float s = f / (2.0f + f);
  float z = s * s;
  float R = (float)(1.0 / 9.0);
  R = fmaf(R, z, (float)(1.0 / 7.0));
  R = fmaf(R, z, (float)(1.0 / 5.0));
  R = fmaf(R, z, (float)(1.0 / 3.0));
  R = R * z;
  float hf = s * f;
  float corr = fmaf(2.0f * s, R, -hf);
  float lm = f + corr;
  float ef = (float)e;
  float res = fmaf(ef, LN2_LO, lm);
  return fmaf(ef, LN2_HI, res);
}

/* exp(x) - 1: Taylor series to degree 8 for |x| < ln2/2, else exp(x) - 1. */
float eo_expm1f(float x) {
  if (fabsf(x) < 0.3465735912322998f) {
    float p = (float)(1.0 / 40320.0);
    p = fmaf(p, x, (float)(1.0 / 5040.0));
    p = fmaf(p, x, (float)(1.0 / 720.0));
    p = fmaf(p, x, (float)(1.0 / 120.0));
    p = fmaf(p, x, (float)(1.0 / 24.0));
    p = fmaf(p, x, (float)(1.0 / 6.0));
    p = fmaf(p, x, 0.5f);
    return fmaf(x * p, x, x);
  }
  return eo_expf(x) - 1.0f;
}

/* log(1+x) for x > -1 by the correction log(u) * x/(u-1), u = 1+x rounded
 * (Goldberg 1991, "What every computer scientist should know about
 * floating-point arithmetic", Theorem 4). */
float eo_log1pf(float x) {
  float u = 1.0f + x;
  if (u == 1.0f) return x;
  return eo_logf(u) * (x / (u - 1.0f));
}

void eo_map_f32(int32_t fn, const float* x, float* y, int64_t count) {
  for (int64_t i = 0; i < count; ++i) {
    switch (fn) {
      case 0: y[i] = eo_expf(x[i]); break;
      case 1: y[i] = eo_logf(x[i]); break;
      case 2: y[i] = eo_expm1f(x[i]); break;
      default: y[i] = eo_log1pf(x[i]); break;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Helpers for exact log-probabilities (Loader 2000, "Fast and accurate     */
/* computation of binomial probabilities"): Stirling error and the          */
/* deviance term bd0, both in float32.                                      */
/* ------------------------------------------------------------------------ */
static float rinv_tab[64];   /* rinv_tab[k] = 1/k rounded, k = 1..63 */
static int rinv_ready = 0;
static void ensure_tables(void) {
  if (rinv_ready) return;
  rinv_tab[0] = 0.0f;
  for (int k = 1; k < 64; ++k) rinv_tab[k] = 1.0f / (float)k;
  rinv_ready = 1;
}

/* log(k!) for 0 <= k <= 9 from the exact float factorial. */
static float lfact_small(int k) {
  float fact = 1.0f;
  for (int j = 2; j <= k; ++j) fact = fact * (float)j;
  return eo_logf(fact);
}

/* delta(k) = log k! - (k log k - k + log(2 pi k)/2), k >= 1. */
static float stirlerr(float k) {
  if (k < 10.0f) {
    float t = (k + 0.5f) * eo_logf(k);
    t = t - k;
    t = t + 0.5f * LN_2PI;
    return lfact_small((int)k) - t;
  }
  /* 1/(12k) - 1/(360k^3) + 1/(1260k^5), nested in r = 1/k (one division) */
  float r = 1.0f / k;
  float r2 = r * r;
  float s = (float)(1.0 / 1260.0) * r2;
  s = (float)(1.0 / 360.0) - s;
  s = s * r2;
  s = (float)(1.0 / 12.0) - s;
  return s * r;
}

/* bd0(x, m) = x log(x/m) + m - x, by its odd series in v = (x-m)/(x+m) when
 * x is near m (five terms: remaining terms below 1e-8 relative); the term of
 * v^(2j+1) carries 1/(2j+1) as a float constant. */
static const float inv_odd[6] = {0.0f, (float)(1.0 / 3.0), (float)(1.0 / 5.0), (float)(1.0 / 7.0),
                                 (float)(1.0 / 9.0), (float)(1.0 / 11.0)};
static float bd0(float x, float m) {
  if (x == 0.0f) return m;
  float d = x - m;
  if (fabsf(d) < 0.1f * (x + m)) {
    float v = d / (x + m);
    float s = d * v;
    float ej = 2.0f * x * v;
    float v2 = v * v;
    for (int j = 1; j <= 5; ++j) {
      ej = ej * v2;
      s = s + ej * inv_odd[j];
    }
    return s;
  }
  return x * eo_logf(x / m) + m - x;
}

/* log of the Poisson(lam) pmf at k. */
static float logpmf_pois(int k, float lam) {
  if (k == 0) return -lam;
  float kf = (float)k;
  if (k < 10) return kf * eo_logf(lam) - lam - lfact_small(k);
  float t = LN_2PI + eo_logf(kf);
  float res = -0.5f * t;
  res = res - stirlerr(kf);
  return res - bd0(kf, lam);
}

/* log of the Binomial(n, p) pmf at k, p <= 1/2, q = 1 - p. */
static float logpmf_binom(int k, int n, float p, float q) {
  float nf = (float)n;
  if (k == 0) return nf * eo_log1pf(-p);
  if (k == n) return nf * eo_logf(p);
  float kf = (float)k, nkf = (float)(n - k);
  float lc = stirlerr(nf) - stirlerr(kf) - stirlerr(nkf) - bd0(kf, nf * p) - bd0(nkf, nf * q);
  float lf = LN_2PI + eo_logf(kf) + eo_log1pf(-(kf / nf));
  return lc - 0.5f * lf;
}

/* ------------------------------------------------------------------------ */
/* Samplers.  Each returns through *err a nonzero code if a rejection loop  */
/* hit the iteration cap (it then returns a defined fallback value).        */
/* ------------------------------------------------------------------------ */

/* Poisson(lam): none drawn if lam <= 0; inversion by sequential search of the
 * cdf for lam < 10; Hoermann's PTRS transformed rejection for lam >= 10
 * (Hoermann 1993, "The transformed rejection method for generating Poisson
 * random variables"). */
static int32_t sample_poisson(float lam, stream_t* st, int* err) {
  if (!(lam > 0.0f)) return 0;
  if (lam < 10.0f) {
    CNT(EOC_POIS_INV);
    float u = next_uniform(st);
    float p = eo_expf(-lam);
    float F = p;
    int32_t k = 0;
    while (u > F) {
      if (k == 63) break;
      k = k + 1;
      CNT(EOC_POIS_INV_ITERS);
      p = (p * lam) * rinv_tab[k];
      float Fn = F + p;
      if (Fn == F) break;
      F = Fn;
    }
    return k;
  }
  CNT(EOC_POIS_PTRS);
  float slam = sqrtf(lam);
  float b = 0.931f + 2.53f * slam;
  float a = -0.059f + 0.02483f * b;
  float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
  float vr = 0.9277f - 3.6224f / (b - 2.0f);
  for (int32_t it = 0; it < g_cap; ++it) {
    CNT(EOC_POIS_PTRS_ITERS);
    float U = next_uniform(st) - 0.5f;
    float V = next_uniform(st);
    float us = 0.5f - fabsf(U);
    float kf = floorf((2.0f * a / us + b) * U + lam + 0.43f);
    if (us >= 0.07f && V <= vr) return (int32_t)kf;
    if (kf < 0.0f || (us < 0.013f && V > us)) continue;
    if (kf > 1.0e9f) continue;
    CNT(EOC_POIS_PTRS_LOGTESTS);
    int32_t k = (int32_t)kf;
    float lhs = eo_logf(V * inv_alpha / (a / (us * us) + b));
    if (lhs <= logpmf_pois(k, lam)) return k;
  }
  *err = EO_ERR_SAMPLER_CAP;
  return (int32_t)floorf(lam);
}

/* Binomial(n, p) for p <= 1/2: inversion for n p < 10, Hoermann's BTRS
 * transformed rejection otherwise (Hoermann 1993, "The generation of binomial
 * random variates"), with the acceptance test on exact log-probabilities. */
static int32_t binom_core(int32_t n, float p, stream_t* st, int* err) {
  float nf = (float)n;
  float np = nf * p;
  float q = 1.0f - p;
  if (np < 10.0f) {
    CNT(EOC_BIN_INV);
    float r = p / q;
    float pk = eo_expf(nf * eo_log1pf(-p));
    float F = pk;
    float u = next_uniform(st);
    int32_t k = 0;
    while (u > F) {
      if (k == n || k == 63) break;
      CNT(EOC_BIN_INV_ITERS);
      pk = ((pk * (float)(n - k)) * r) * rinv_tab[k + 1];
      k = k + 1;
      float Fn = F + pk;
      if (Fn == F) break;
      F = Fn;
    }
    return k;
  }
  CNT(EOC_BIN_BTRS);
  float spq = sqrtf(np * q);
  float b = 1.15f + 2.53f * spq;
  float a = -0.0873f + 0.0248f * b + 0.01f * p;
  float c = np + 0.5f;
  float vr = 0.92f - 4.2f / b;
  float alpha = (2.83f + 5.1f / b) * spq;
  int32_t m = (int32_t)floorf((nf + 1.0f) * p);
  if (m > n) m = n;
  float lpm = logpmf_binom(m, n, p, q);
  for (int32_t it = 0; it < g_cap; ++it) {
    CNT(EOC_BIN_BTRS_ITERS);
    float u = next_uniform(st) - 0.5f;
    float v = next_uniform(st);
    float us = 0.5f - fabsf(u);
    float kf = floorf((2.0f * a / us + b) * u + c);
    if (kf < 0.0f || kf > nf) continue;
    int32_t k = (int32_t)kf;
    if (us >= 0.07f && v <= vr) return k;
    CNT(EOC_BIN_BTRS_LOGTESTS);
    float lv = eo_logf(v * alpha / (a / (us * us) + b));
    if (lv <= logpmf_binom(k, n, p, q) - lpm) return k;
  }
  *err = EO_ERR_SAMPLER_CAP;
  return (int32_t)floorf(np);
}

/* Binomial(n, p): zero draws if n = 0 or p <= 0 ("return zero if the first
 * argument is zero", Appendix A); n if p >= 1; symmetric reduction for
 * p > 1/2 (1 - p is exact there). */
static int32_t sample_binomial(int32_t n, float p, stream_t* st, int* err) {
  if (n <= 0 || !(p > 0.0f)) return 0;
  if (p >= 1.0f) return n;
  if (p > 0.5f) return n - binom_core(n, 1.0f - p, st, err);
  return binom_core(n, p, st, err);
}

/* Standard normal by Marsaglia's polar method (one of the pair is used). */
static float sample_normal(stream_t* st, int* err) {
  for (int32_t it = 0; it < g_cap; ++it) {
    CNT(EOC_NORMAL_ITERS);
    float v1 = 2.0f * next_uniform(st) - 1.0f;
    float v2 = 2.0f * next_uniform(st) - 1.0f;
    float s = v1 * v1 + v2 * v2;
    if (s < 1.0f) {
      float t = (-2.0f * eo_logf(s)) / s;
      return v1 * sqrtf(t);
    }
  }
  *err = EO_ERR_SAMPLER_CAP;
  return 0.0f;
}

/* Erlang(k, rate) = Gamma(k)/rate.  k <= 8: minus the log of products of at
 * most four uniforms, summed; k > 8: Marsaglia & Tsang (2000), "A simple
 * method for generating gamma variables". */
static float sample_erlang(int32_t k, float rate, stream_t* st, int* err) {
  if (k <= 0) return 0.0f;
  if (k <= 8) {
    CNT(EOC_GAMMA_SMALL);
    float S = 0.0f;
    int32_t rem = k;
    while (rem > 0) {
      int32_t g = rem < 4 ? rem : 4;
      float prod = next_uniform(st);
      for (int32_t j = 1; j < g; ++j) prod = prod * next_uniform(st);
      CNT(EOC_GAMMA_SMALL_LOGS);
      S = S - eo_logf(prod);
      rem = rem - g;
    }
    return S / rate;
  }
  CNT(EOC_GAMMA_MT);
  float d = (float)k - (float)(1.0 / 3.0);
  float cc = 1.0f / sqrtf(9.0f * d);
  for (int32_t it = 0; it < g_cap; ++it) {
    CNT(EOC_GAMMA_MT_ITERS);
    float x = sample_normal(st, err);
    float v = 1.0f + cc * x;
    if (v <= 0.0f) continue;
    v = v * v * v;
    float u = next_uniform(st);
    float x2 = x * x;
    if (u < 1.0f - 0.0331f * (x2 * x2)) return d * v / rate;
    if (eo_logf(u) < 0.5f * x2 + d * ((1.0f - v) + eo_logf(v))) return d * v / rate;
  }
  *err = EO_ERR_SAMPLER_CAP;
  return (float)k / rate;
}

/* GenerateDeparture(x, m, mu, h): Lemma 1 / Algorithm 1.
 *   x <= m : Binomial(x, 1 - e^{-mu h})
 *   x >  m : T ~ Erlang(x - m, m mu);
 *            T >  h : Binomial(x - m - 1, h / T)
 *            T <= h : (x - m) + Binomial(m, 1 - e^{-mu (h - T)})
 * p0 = 1 - e^{-mu h} is passed in (computed once per station). */
static int32_t departure(int32_t x, int32_t m, float mu, float h, float p0, float muh,
                         stream_t* st, int* err, float* score_mu) {
  if (g_dep_mode == 1 || (g_dep_mode == 2 && x > m)) {
    /* Eq. (1): the busy count frozen at b = min(x, m) over the step,
       D = min(x, S) with S ~ Poisson(b mu h) (Eq. (2) keeps this for x > m) */
    int32_t b = x < m ? x : m;
    int32_t S = sample_poisson((float)b * muh, st, err);
    if (score_mu) *score_mu = 0.0f;
    return S < x ? S : x;
  }
  if (x <= m) {
    CNT(EOC_DEP_LE_M);
    int32_t k = sample_binomial(x, p0, st, err);
    /* d/dmu log Bin(k; x, p0(mu)), dp0/dmu = h (1 - p0):  h (k/p0 - x) */
    if (score_mu) *score_mu = h * ((k > 0 ? (float)k / p0 : 0.0f) - (float)x);
    return k;
  }
  float rate = (float)m * mu;
  /* T from the Erlang stream (purpose 2) of this station, step and replication */
  stream_t es;
  stream_sibling(&es, st, 2u);
  float T = sample_erlang(x - m, rate, &es, err);
  /* d/dmu log of the Erlang(x - m, m mu) density at T:  (x - m)/mu - m T */
  float te = (float)(x - m) / mu - (float)m * T;
  if (T > h) {
    CNT(EOC_DEP_T_GT_H);
    if (score_mu) *score_mu = te;  /* Bin(x - m - 1, h/T) does not depend on mu */
    return sample_binomial(x - m - 1, h / T, st, err);
  }
  CNT(EOC_DEP_T_LE_H);
  float p = -eo_expm1f(-(mu * (h - T)));
  int32_t k2 = sample_binomial(m, p, st, err);
  /* d/dmu log Bin(k2; m, p(mu)), dp/dmu = (h - T)(1 - p) */
  if (score_mu) *score_mu = te + (h - T) * ((k2 > 0 ? (float)k2 / p : 0.0f) - (float)m);
  return (x - m) + k2;
}

/* Routing (Sec. 2.2): (R_i1..R_in, R_i_exit) ~ Multinomial(D, (p_i., p_i_exit)),
 * drawn as sequential conditional binomials along the CSR row:
 * R_e ~ Binomial(rem, qc_e), rem -= R_e; the exit count is what remains. */
static int32_t route(int32_t D, int32_t e0, int32_t e1, const float* qc, int32_t* Redge,
                     stream_t* st, int* err) {
  int32_t rem = D;
  for (int32_t e = e0; e < e1; ++e) {
    int32_t r = 0;
    if (rem > 0) { CNT(EOC_ROUTE_BINOMIALS); r = sample_binomial(rem, qc[e], st, err); }
    Redge[e] = r;
    rem = rem - r;
  }
  return rem;
}

/* Conditional split probabilities qc_e = p_e / (p_exit + sum_{e' >= e} p_e'),
 * in double, clamped to [0, 1], then rounded to float.  A row whose exit
 * probability is below 1e-12 is treated as exit-free, so its last edge takes
 * everything that remains (qc = 1 exactly). */
static void cond_probs(const eo_net* net, float* qc) {
  for (int32_t i = 0; i < net->n; ++i) {
    int32_t e0 = net->row_ptr[i], e1 = net->row_ptr[i + 1];
    double rowsum = 0.0;
    for (int32_t e = e0; e < e1; ++e) rowsum += net->prob[e];
    double pexit = 1.0 - rowsum;
    if (pexit < 1e-12) pexit = 0.0;
    double suffix = pexit;
    for (int32_t e = e1 - 1; e >= e0; --e) {
      suffix += net->prob[e];
      double q = suffix > 0.0 ? net->prob[e] / suffix : 0.0;
      if (q < 0.0) q = 0.0;
      if (q > 1.0) q = 1.0;
      qc[e] = (float)q;
    }
  }
}

/* Aggregated external-arrival mean over step tau (Sec. 2.1.1):
 * Lambda = integral of lambda_i(u) over ((tau-1) dt, tau dt]. */
static double interval_rate(const eo_net* net, int32_t i, int64_t tau, double dt) {
  double t0 = (double)(tau - 1) * dt;
  double t1 = (double)tau * dt;
  if (net->arr_kind == EO_ARR_SINUSOID) {
    double om = 6.283185307179586 / net->period;
    double lam = net->w[i] * net->a *
                 ((t1 - t0) + net->b * (cos(om * t0 + net->phase) - cos(om * t1 + net->phase)) / om);
    return lam > 0.0 ? lam : 0.0;
  }
  if (net->arr_kind == EO_ARR_TABLE) {
    /* exact integral of the piecewise-linear interpolant, segment by segment */
    const int32_t J = net->table_len, n = net->n;
    const double td = net->tab_dt;
    double total = 0.0;
    double a = t0;
    while (a < t1) {
      double j_real = floor(a / td);
      int64_t j = (int64_t)j_real;
      double seg_end = (double)(j + 1) * td;
      double b = seg_end < t1 ? seg_end : t1;
      if (b <= a) b = t1; /* guard against a / td rounding at a grid point */
      double la, lb;
      if (j >= J - 1) {
        la = lb = net->table[(int64_t)(J - 1) * n + i];
      } else {
        double y0 = net->table[j * n + i], y1 = net->table[(j + 1) * n + i];
        double ta = (double)j * td;
        la = y0 + (y1 - y0) * ((a - ta) / td);
        lb = y0 + (y1 - y0) * ((b - ta) / td);
      }
      total += (b - a) * (la + lb) * 0.5;
      a = b;
    }
    return total > 0.0 ? total : 0.0;
  }
  return 0.0;
}

/* d Lambda / d (a, b, phase) for the sinusoid (zero for other kinds, and
 * where Lambda was clamped at zero). */
static void interval_rate_grad(const eo_net* net, int32_t i, int64_t tau, double dt, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (net->arr_kind != EO_ARR_SINUSOID) return;
  if (!(interval_rate(net, i, tau, dt) > 0.0)) return;
  double t0 = (double)(tau - 1) * dt;
  double t1 = (double)tau * dt;
  double om = 6.283185307179586 / net->period;
  double c0 = cos(om * t0 + net->phase), c1 = cos(om * t1 + net->phase);
  double s0 = sin(om * t0 + net->phase), s1 = sin(om * t1 + net->phase);
  g[0] = net->w[i] * ((t1 - t0) + net->b * (c0 - c1) / om);
  g[1] = net->w[i] * net->a * ((c0 - c1) / om);
  g[2] = net->w[i] * net->a * net->b * ((s1 - s0) / om);
}

/* Servers of every station during step tau (Sec. 2.1.2): the staffing
 * schedule at the step's start time (tau - 1) dt, or the constant m_i. */
static const int32_t* servers_of_step(const eo_net* net, int64_t tau, double dt) {
  if (!net->sv_table) return net->servers;
  int64_t j = (int64_t)floor((double)(tau - 1) * dt / net->sv_dt);
  if (j > net->sv_len - 1) j = net->sv_len - 1;
  return net->sv_table + j * net->n;
}

int64_t eo_num_steps(double dt, double T) {
  double k = ceil(T / dt - 1e-9);
  return k < 1.0 ? 1 : (int64_t)k;
}

/* Per-draw score terms of one unit: the departure's mu_i term, and for an
 * external-arrival draw (lam > 0) (A/lam - 1) dLambda/dtheta. */
static void accumulate_scores(int32_t i, float smu, int32_t A, float lam, const float* dl,
                              double* mu_acc, double* th_acc) {
  mu_acc[i] += (double)smu;
  if (lam > 0.0f) {
    float g = (float)A / lam - 1.0f;
    for (int k = 0; k < 3; ++k) th_acc[3 * i + k] += (double)(g * dl[k]);
  }
}

/* Topological order by Kahn's algorithm (smallest ready index first). */
static int topo_order(const eo_net* net, int32_t* order) {
  const int32_t n = net->n;
  int32_t* indeg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* ready = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t nready = 0, count = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) indeg[net->col[e]]++;
  for (int32_t i = 0; i < n; ++i)
    if (indeg[i] == 0) ready[nready++] = i;
  while (nready > 0) {
    /* take the smallest ready index */
    int32_t best = 0;
    for (int32_t j = 1; j < nready; ++j)
      if (ready[j] < ready[best]) best = j;
    int32_t i = ready[best];
    ready[best] = ready[--nready];
    order[count++] = i;
    for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e)
      if (--indeg[net->col[e]] == 0) ready[nready++] = net->col[e];
  }
  free(indeg);
  free(ready);
  return count == n ? EO_OK : EO_ERR_NOT_FEEDFORWARD;
}

static int validate(const eo_net* net) {
  if (!net || net->n <= 0 || !net->row_ptr || !net->servers || !net->mu) return EO_ERR_ARG;
  if (net->row_ptr[0] != 0) return EO_ERR_ARG;
  for (int32_t i = 0; i < net->n; ++i) {
    if (net->row_ptr[i + 1] < net->row_ptr[i]) return EO_ERR_ARG;
    if (net->servers[i] < 1 || !(net->mu[i] > 0.0) || !isfinite(net->mu[i])) return EO_ERR_ARG;
    double s = 0.0;
    for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) {
      if (net->col[e] < 0 || net->col[e] >= net->n) return EO_ERR_ARG;
      if (!(net->prob[e] >= 0.0 && net->prob[e] <= 1.0)) return EO_ERR_ARG;
      s += net->prob[e];
    }
    if (s > 1.0 + 1e-12) return EO_ERR_ARG;
  }
  if (net->arr_kind == EO_ARR_SINUSOID && (!net->w || !(net->period > 0.0))) return EO_ERR_ARG;
  if (net->sv_table) {
    if (net->sv_len < 1 || !(net->sv_dt > 0.0)) return EO_ERR_ARG;
    for (int64_t k = 0; k < (int64_t)net->sv_len * net->n; ++k)
      if (net->sv_table[k] < 1) return EO_ERR_ARG;
  }
  if (net->arr_kind == EO_ARR_TABLE && (!net->table || net->table_len < 1 || !(net->tab_dt > 0.0)))
    return EO_ERR_ARG;
  return EO_OK;
}

/* The time loop of both schemes; with `scores` != NULL also the score
 * S_r = d log p(path) / d(mu_1..mu_n, a, b, phase) of every replication
 * ([R][n+3] doubles): float32 terms per draw, float64 sums -- mu_i terms in
 * step order, sinusoid terms per external station in step order, then over
 * those stations in index order. */
static int simulate_impl(const eo_net* net, int32_t scheme, double dt, double T, int64_t R,
                         uint64_t seed, int64_t rep_begin, int64_t* stats, int32_t* trace_N,
                         int32_t* trace_D, int32_t* trace_A, int32_t* trace_R, double* scores,
                         int64_t tau0, const int32_t* N_in, int32_t* N_out) {
  int rc = validate(net);
  if (rc) return rc;
  if (!(dt > 0.0) || !(T > 0.0) || R < 0 || rep_begin < 0 || !stats) return EO_ERR_ARG;
  if (scheme != EO_BACKWARD && scheme != EO_FORWARD) return EO_ERR_ARG;
  ensure_tables();
  const int32_t n = net->n;
  const int32_t E = net->row_ptr[n];
  const int64_t K = eo_num_steps(dt, T);
  if (tau0 < 0 || tau0 > K) return EO_ERR_ARG;

  int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  rc = topo_order(net, order);
  if (rc) { free(order); return rc; }

  /* per-station float parameters */
  float* mu_f = (float*)malloc((size_t)n * sizeof(float));
  float* p0 = (float*)malloc((size_t)n * sizeof(float));
  float* muh = (float*)malloc((size_t)n * sizeof(float));
  const float h_f = (float)dt;
  for (int32_t i = 0; i < n; ++i) {
    mu_f[i] = (float)net->mu[i];
    float y = (float)(net->mu[i] * dt);
    muh[i] = y;
    p0[i] = -eo_expm1f(-y);
  }
  float* qc = (float*)malloc((size_t)(E > 0 ? E : 1) * sizeof(float));
  cond_probs(net, qc);

  /* reverse graph (CSC): edges into each station */
  int32_t* in_ptr = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* in_edge = (int32_t*)malloc((size_t)(E > 0 ? E : 1) * sizeof(int32_t));
  for (int32_t e = 0; e < E; ++e) in_ptr[net->col[e] + 1]++;
  for (int32_t i = 0; i < n; ++i) in_ptr[i + 1] += in_ptr[i];
  {
    int32_t* fill = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i)
      for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) {
        int32_t j = net->col[e];
        in_edge[in_ptr[j] + fill[j]++] = e;
      }
    free(fill);
  }

  /* Lambda table, double -> float, [K][n]; steps of the perturbation window
     (eo_set_arrival_window) scaled in double before the rounding */
  float* lam = (float*)malloc((size_t)K * (size_t)n * sizeof(float));
  for (int64_t tau = 1; tau <= K; ++tau)
    for (int32_t i = 0; i < n; ++i) {
      double L = interval_rate(net, i, tau, dt);
      if (tau >= g_win_lo && tau <= g_win_hi) L = L * g_win_factor;
      lam[(tau - 1) * n + i] = (float)L;
    }

  float* dlam = NULL;           /* [K][n][3] */
  double* mu_acc = NULL;        /* [n] */
  double* th_acc = NULL;        /* [n][3] */
  if (scores) {
    dlam = (float*)malloc((size_t)K * (size_t)n * 3 * sizeof(float));
    for (int64_t tau = 1; tau <= K; ++tau)
      for (int32_t i = 0; i < n; ++i) {
        double g[3];
        interval_rate_grad(net, i, tau, dt, g);
        for (int k = 0; k < 3; ++k) dlam[((tau - 1) * n + i) * 3 + k] = (float)g[k];
      }
    mu_acc = (double*)malloc((size_t)n * sizeof(double));
    th_acc = (double*)malloc((size_t)n * 3 * sizeof(double));
  }

  int64_t* st_station = stats;            /* [n][5] */
  int64_t* st_rep = stats + 5 * (int64_t)n; /* [R][4] */
  int64_t* st_NK = st_rep + 4 * R;        /* [n]    */
  memset(stats, 0, (size_t)(6 * (int64_t)n + 4 * R) * sizeof(int64_t));

  int32_t* N = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* D = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* X = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* A = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* Redge = (int32_t*)calloc((size_t)(E > 0 ? E : 1), sizeof(int32_t));

  int err = 0;
  for (int64_t r = 0; r < R && !err; ++r) {
    const uint32_t rep = (uint32_t)(rep_begin + r);
    for (int32_t i = 0; i < n; ++i) N[i] = N_in ? N_in[(int64_t)i * R + r] : net->N0 ? net->N0[i] : 0;
    if (scores)
      for (int32_t i = 0; i < n; ++i) {
        mu_acc[i] = 0.0;
        th_acc[3 * i] = th_acc[3 * i + 1] = th_acc[3 * i + 2] = 0.0;
      }
    for (int64_t tau = tau0 + 1; tau <= K && !err; ++tau) {
      const float* lam_t = lam + (tau - 1) * n;
      const int32_t* m_t = servers_of_step(net, tau, dt);
      if (scheme == EO_BACKWARD) {
        /* Sec. 2.2 backward tasks 1-3 for every node from N_{tau-1} ... */
        for (int32_t i = 0; i < n; ++i) {
          stream_t svc, arr;
          stream_init(&svc, seed, 1u, (uint32_t)i, (uint32_t)tau, rep);
          float smu = 0.0f;
          D[i] = departure(N[i], m_t[i], mu_f[i], h_f, p0[i], muh[i], &svc, &err, &smu);
          X[i] = route(D[i], net->row_ptr[i], net->row_ptr[i + 1], qc, Redge, &svc, &err);
          stream_init(&arr, seed, 0u, (uint32_t)i, (uint32_t)tau, rep);
          A[i] = sample_poisson(lam_t[i], &arr, &err);
          if (scores) accumulate_scores(i, smu, A[i], lam_t[i], dlam + ((tau - 1) * n + i) * 3, mu_acc, th_acc);
        }
        /* ... then task 4 once every node has routed (Algorithm 2). */
        for (int32_t i = 0; i < n; ++i) {
          int64_t ain = 0;
          for (int32_t k = in_ptr[i]; k < in_ptr[i + 1]; ++k) { ain += Redge[in_edge[k]]; CNT(EOC_GATHER_EDGES); }
          int64_t nn = (int64_t)N[i] - D[i] + A[i] + ain;
          if (nn > (1 << 30)) { err = EO_ERR_OVERFLOW; nn = 1 << 30; }
          N[i] = (int32_t)nn;
          CNT(EOC_UNITS);
        }
      } else {
        /* Sec. 2.2 forward tasks node by node in flow order (Algorithm 3). */
        for (int32_t oi = 0; oi < n; ++oi) {
          const int32_t i = order[oi];
          stream_t svc, arr;
          stream_init(&arr, seed, 0u, (uint32_t)i, (uint32_t)tau, rep);
          A[i] = sample_poisson(lam_t[i], &arr, &err);
          int64_t ain = 0;
          for (int32_t k = in_ptr[i]; k < in_ptr[i + 1]; ++k) { ain += Redge[in_edge[k]]; CNT(EOC_GATHER_EDGES); }
          int64_t y = (int64_t)N[i] + A[i] + ain;
          if (y > (1 << 30)) { err = EO_ERR_OVERFLOW; y = 1 << 30; }
          stream_init(&svc, seed, 1u, (uint32_t)i, (uint32_t)tau, rep);
          float smu = 0.0f;
          D[i] = departure((int32_t)y, m_t[i], mu_f[i], h_f, p0[i], muh[i], &svc, &err, &smu);
          if (scores) accumulate_scores(i, smu, A[i], lam_t[i], dlam + ((tau - 1) * n + i) * 3, mu_acc, th_acc);
          N[i] = (int32_t)y - D[i];
          X[i] = route(D[i], net->row_ptr[i], net->row_ptr[i + 1], qc, Redge, &svc, &err);
          CNT(EOC_UNITS);
        }
      }
      /* streaming statistics over post-update states */
      int64_t* sr = st_rep + 4 * r;
      for (int32_t i = 0; i < n; ++i) {
        int64_t* ss = st_station + 5 * (int64_t)i;
        ss[0] += N[i];
        ss[1] += N[i] < m_t[i] ? N[i] : m_t[i];
        ss[2] += D[i];
        ss[3] += X[i];
        ss[4] += A[i];
        sr[0] += N[i];
        sr[1] += D[i];
        sr[2] += X[i];
        sr[3] += A[i];
      }
      if (trace_N || trace_D || trace_A) {
        for (int32_t i = 0; i < n; ++i) {
          int64_t idx = ((tau - 1) * n + i) * R + r;
          if (trace_N) trace_N[idx] = N[i];
          if (trace_D) trace_D[idx] = D[i];
          if (trace_A) trace_A[idx] = A[i];
        }
      }
      if (trace_R)
        for (int32_t e = 0; e < E; ++e) trace_R[((tau - 1) * E + e) * R + r] = Redge[e];
    }
    for (int32_t i = 0; i < n; ++i) st_NK[i] += N[i];
    if (N_out)
      for (int32_t i = 0; i < n; ++i) N_out[(int64_t)i * R + r] = N[i];
    if (scores) {
      double* sr = scores + r * (int64_t)(n + 3);
      for (int32_t i = 0; i < n; ++i) sr[i] = mu_acc[i];
      sr[n] = sr[n + 1] = sr[n + 2] = 0.0;
      for (int32_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) sr[n + k] += th_acc[3 * i + k];
    }
  }
  free(dlam); free(mu_acc); free(th_acc);

  free(order); free(mu_f); free(p0); free(muh); free(qc); free(in_ptr); free(in_edge); free(lam);
  free(N); free(D); free(X); free(A); free(Redge);
  return err;
}

/* ------------------------------------------------------------------------ */
/* Direct sampler access for the distribution tests.                        */
/* ------------------------------------------------------------------------ */
int eo_draw_poisson(float lam, uint64_t seed, int64_t count, int32_t* out) {
  ensure_tables();
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    out[j] = sample_poisson(lam, &st, &err);
  }
  return err;
}

int eo_draw_binomial(int32_t n, float p, uint64_t seed, int64_t count, int32_t* out) {
  ensure_tables();
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    out[j] = sample_binomial(n, p, &st, &err);
  }
  return err;
}

int eo_draw_gamma(int32_t k, float rate, uint64_t seed, int64_t count, float* out) {
  ensure_tables();
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    out[j] = sample_erlang(k, rate, &st, &err);
  }
  return err;
}

int eo_draw_normal(uint64_t seed, int64_t count, float* out) {
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    out[j] = sample_normal(&st, &err);
  }
  return err;
}

int eo_draw_departure(int32_t x, int32_t m, double mu, double h, uint64_t seed, int64_t count,
                      int32_t* out) {
  ensure_tables();
  if (m < 1 || !(mu > 0.0) || !(h > 0.0) || x < 0) return EO_ERR_ARG;
  float mu_f = (float)mu, h_f = (float)h;
  float p0 = -eo_expm1f(-(float)(mu * h));
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    out[j] = departure(x, m, mu_f, h_f, p0, (float)(mu * h), &st, &err, NULL);
  }
  return err;
}

int eo_draw_route(int32_t D, int32_t deg, const double* prob, uint64_t seed, int64_t count,
                  int32_t* out) {
  ensure_tables();
  if (deg < 0 || D < 0) return EO_ERR_ARG;
  int32_t row_ptr[2] = {0, deg};
  int32_t one_server = 1;
  double one_mu = 1.0;
  int32_t* col = (int32_t*)calloc((size_t)(deg > 0 ? deg : 1), sizeof(int32_t));
  eo_net net;
  memset(&net, 0, sizeof net);
  net.n = 1; net.row_ptr = row_ptr; net.col = col; net.prob = prob;
  net.servers = &one_server; net.mu = &one_mu;
  float* qc = (float*)malloc((size_t)(deg > 0 ? deg : 1) * sizeof(float));
  cond_probs(&net, qc);
  int32_t* Redge = (int32_t*)malloc((size_t)(deg > 0 ? deg : 1) * sizeof(int32_t));
  int err = 0;
  for (int64_t j = 0; j < count; ++j) {
    stream_t st;
    stream_init(&st, seed, 1u, 0u, 0u, (uint32_t)j);
    int32_t ex = route(D, 0, deg, qc, Redge, &st, &err);
    for (int32_t e = 0; e < deg; ++e) out[j * (deg + 1) + e] = Redge[e];
    out[j * (deg + 1) + deg] = ex;
  }
  free(col); free(qc); free(Redge);
  return err;
}

void eo_uniforms(uint64_t seed, uint32_t purpose, uint32_t station, uint32_t step, uint32_t rep,
                 int64_t count, float* out) {
  stream_t st;
  stream_init(&st, seed, purpose, station, step, rep);
  for (int64_t j = 0; j < count; ++j) out[j] = next_uniform(&st);
}

int eo_simulate(const eo_net* net, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
                int64_t rep_begin, int64_t* stats, int32_t* trace_N, int32_t* trace_D,
                int32_t* trace_A) {
  return simulate_impl(net, scheme, dt, T, R, seed, rep_begin, stats, trace_N, trace_D, trace_A,
                       NULL, NULL, 0, NULL, NULL);
}

/* Checkpoint / resume: the steps tau0+1..K from the state N_in = N_tau0
 * ([n][R], replication fastest; NULL = N0 of the network), keyed exactly as
 * in the uninterrupted run, so the two halves of a split run reproduce it.
 * N_out ([n][R] or NULL) receives N_K. */
int eo_simulate_resume(const eo_net* net, int32_t scheme, double dt, double T, int64_t R,
                       uint64_t seed, int64_t rep_begin, int64_t tau0, const int32_t* N_in,
                       int32_t* N_out, int64_t* stats) {
  return simulate_impl(net, scheme, dt, T, R, seed, rep_begin, stats, NULL, NULL, NULL, NULL, NULL,
                       tau0, N_in, N_out);
}

/* Likelihood-ratio (score-function) gradient of the two measures
 *   L1_r = dt * sum_{tau, i} N_{tau,i}   (time-integrated total count)
 *   L2_r = sum_{tau, i} D_{tau,i}        (total departures)
 * with respect to (mu_1..mu_n, a, b, phase):  grad[m][c] = mean_r L_m(r) S_r[c],
 * value[m] = mean_r L_m(r), grad_var[m][c] = variance of that mean.  Sums over
 * replications run in blocks of 32 consecutive replications (ascending inside
 * a block), then over blocks in ascending order.  scores_out (may be NULL)
 * receives S_r, [R][n+3]. */
int eo_grad(const eo_net* net, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
            int64_t rep_begin, double* scores_out, double* grad, double* value, double* grad_var) {
  if (R < 1 || !grad || !value || g_dep_mode != 0) return EO_ERR_ARG;
  const int32_t n = net->n;
  const int64_t C = n + 3;
  int64_t* stats = (int64_t*)malloc((size_t)(6 * (int64_t)n + 4 * R) * sizeof(int64_t));
  double* sc = scores_out ? scores_out : (double*)malloc((size_t)(R * C) * sizeof(double));
  int rc = simulate_impl(net, scheme, dt, T, R, seed, rep_begin, stats, NULL, NULL, NULL, NULL, sc,
                         0, NULL, NULL);
  if (rc == EO_OK) {
    const int64_t* rp = stats + 5 * (int64_t)n;
    for (int m = 0; m < 2; ++m) {
      double vsum = 0.0;
      for (int64_t b0 = 0; b0 < R; b0 += 32) {
        double part = 0.0;
        for (int64_t r = b0; r < R && r < b0 + 32; ++r)
          part += m == 0 ? dt * (double)rp[4 * r] : (double)rp[4 * r + 1];
        vsum += part;
      }
      value[m] = vsum / (double)R;
      /* centred estimator: (L - mean L) S, same expectation since E[S] = 0 */
      const double Lbar = g_grad_center ? value[m] : 0.0;
      for (int64_t c = 0; c < C; ++c) {
        double s = 0.0, ss = 0.0;
        for (int64_t b0 = 0; b0 < R; b0 += 32) {
          double part = 0.0, part2 = 0.0;
          for (int64_t r = b0; r < R && r < b0 + 32; ++r) {
            double L = m == 0 ? dt * (double)rp[4 * r] : (double)rp[4 * r + 1];
            double x = (g_grad_center ? L - Lbar : L) * sc[r * C + c];
            part += x;
            part2 += x * x;
          }
          s += part;
          ss += part2;
        }
        double g = s / (double)R;
        grad[m * C + c] = g;
        if (grad_var)
          grad_var[m * C + c] = R > 1 ? (ss - (double)R * g * g) / ((double)R * (double)(R - 1)) : 0.0;
      }
    }
  }
  if (!scores_out) free(sc);
  free(stats);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sojourn time of a tagged customer: Sec. 6, Algorithm 4, with the          */
/* conditional probability of Lemma 3.                                      */
/* ------------------------------------------------------------------------ */

/* b^k for an integer k >= 0 by binary powering (the multiplications in a
 * fixed order, so both sides of the parity check round identically). */
static float pow_int(float b, int32_t k) {
  float r = 1.0f;
  while (k > 0) {
    if (k & 1) r = r * b;
    b = b * b;
    k >>= 1;
  }
  return r;
}

/* Lemma 3: a server busy with the tagged customer at the start of a step is
 * still busy with it at the end, given that the step's departure draw had
 * input x (customers at the station) and output d (m servers):
 *   x <= m          : (x - d) / x
 *   m < x <= m + d  : ((m-1)/m)^(x-m) (x - d) / m
 *   x > m + d       : ((m-1)/m)^d
 * d = 0 gives 1 in every case (also for an x = 0 that a sample path can show
 * at the tagged customer's station: nothing left, so nothing ends service). */
float eo_sojourn_pstay(int32_t x, int32_t d, int32_t m) {
  if (d <= 0) return 1.0f;
  if (x <= m) return (float)(x - d) / (float)x;
  float q = (float)(m - 1) / (float)m;
  if (x <= m + d) return pow_int(q, x - m) * ((float)(x - d) / (float)m);
  return pow_int(q, d);
}

/* Algorithm 4 over stored sample paths.  The paths are simulated first with
 * the given scheme (N_tau, D_tau and the routed counts R_tau,e of every step
 * are kept); then, for every replication r and tagged customer s, the
 * algorithm runs on path r:
 *   Setup    at station i after step tau: position p = max(N_tau,i, 1); if
 *            p > m_i wait, else serve.
 *   Waiting  eta = min{j >= 1 : p - D_tau+1,i - ... - D_tau+j,i <= m_i};
 *            T += eta h, tau += eta; then serve.
 *   Service  step tau+1: stay with probability Lemma 3 (x, d) where d =
 *            D_tau+1,i and x is the input of that departure draw (N_tau,i for
 *            the backward scheme, N_tau+1,i + D_tau+1,i for the forward one);
 *            T += h, tau += 1; on leaving, go to station j with probability
 *            R_tau,ij / D_tau,i or exit with the remaining mass.
 * m_i is the staffing of the step whose values are read.  Random choices use
 * the stream (seed, purpose 3, station slot s, step tau, replication): its
 * first uniform decides the stay (stay iff u < p_stay), its second word w
 * picks the departing customer k = floor(w d / 2^32) among the d departures,
 * which go, in CSR order, to the edges' destinations and then to the exit.
 * out[r * samples + s] = the sojourn in steps (T / h) if the customer left
 * by step K, else -(steps accounted up to step K) (censored; <= 0). */
int eo_sojourn(const eo_net* net, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
               int64_t rep_begin, int32_t station, int64_t tau0, int32_t samples, int32_t* out,
               int64_t* stats) {
  int rc = validate(net);
  if (rc) return rc;
  const int32_t n = net->n;
  const int32_t E = net->row_ptr[n];
  const int64_t K = eo_num_steps(dt, T);
  if (!(dt > 0.0) || !(T > 0.0) || R < 0 || samples < 1 || !out) return EO_ERR_ARG;
  if (station < 0 || station >= n || tau0 < 1 || tau0 > K) return EO_ERR_ARG;
  const size_t cells = (size_t)K * (size_t)n * (size_t)(R > 0 ? R : 1);
  int32_t* tN = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* tD = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* tR = (int32_t*)malloc((size_t)K * (size_t)(E > 0 ? E : 1) * (size_t)(R > 0 ? R : 1) * sizeof(int32_t));
  int64_t* st = stats ? stats : (int64_t*)malloc((size_t)(6 * (int64_t)n + 4 * R) * sizeof(int64_t));
  if (!tN || !tD || !tR || !st) {
    free(tN); free(tD); free(tR); if (!stats) free(st);
    return EO_ERR_ARG;
  }
  rc = simulate_impl(net, scheme, dt, T, R, seed, rep_begin, st, tN, tD, NULL, tR, NULL, 0, NULL,
                     NULL);
  /* path values: step tau in 1..K, station i, replication r */
#define PN(tau, i) tN[(((tau) - 1) * n + (i)) * R + r]
#define PD(tau, i) tD[(((tau) - 1) * n + (i)) * R + r]
#define PR(tau, e) tR[(((tau) - 1) * E + (e)) * R + r]
  for (int64_t r = 0; r < R && rc == EO_OK; ++r) {
    const uint32_t rep = (uint32_t)(rep_begin + r);
    for (int32_t s = 0; s < samples; ++s) {
      int32_t i = station;
      int64_t tau = tau0;
      int64_t steps = 0;
      int done = 0;
      while (!done) {
        /* Setup step */
        int32_t pos = PN(tau, i);
        if (pos < 1) pos = 1;
        if (pos > servers_of_step(net, tau, dt)[i]) {
          /* Waiting step: eta steps until at most m_i are ahead of or at the
             customer's place */
          int64_t j = 0;
          int64_t left = pos;
          int reached = 0;
          while (tau + j + 1 <= K) {
            ++j;
            left -= PD(tau + j, i);
            if (left <= servers_of_step(net, tau + j, dt)[i]) { reached = 1; break; }
          }
          steps += j;
          tau += j;
          if (!reached) break; /* censored while waiting */
        }
        /* Service step, repeated while the customer stays */
        for (;;) {
          if (tau + 1 > K) { done = -1; break; } /* censored in service */
          const int64_t t1 = tau + 1;
          const int32_t d = PD(t1, i);
          const int32_t x = scheme == EO_BACKWARD ? PN(tau, i) : PN(t1, i) + d;
          const float ps = eo_sojourn_pstay(x, d, servers_of_step(net, t1, dt)[i]);
          stream_t cs;
          stream_init(&cs, seed, 3u, (uint32_t)s, (uint32_t)t1, rep);
          const float u = next_uniform(&cs);
          const uint32_t w = next_word(&cs);
          steps += 1;
          tau = t1;
          if (u < ps) continue; /* I = 1: still in service */
          /* I = 0: the customer is one of the d departures; its destination
             follows the step's routed counts */
          uint32_t k = (uint32_t)(((uint64_t)w * (uint64_t)(uint32_t)d) >> 32);
          int32_t next = -1;
          for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) {
            const uint32_t v = (uint32_t)PR(t1, e);
            if (k < v) { next = net->col[e]; break; }
            k -= v;
          }
          if (next < 0) { done = 1; break; } /* exit: sojourn complete */
          i = next;
          break; /* back to the Setup step at the new station */
        }
      }
      out[r * samples + s] = done == 1 ? (int32_t)steps : -(int32_t)steps;
    }
  }
#undef PN
#undef PD
#undef PR
  free(tN); free(tD); free(tR);
  if (!stats) free(st);
  return rc;
}
