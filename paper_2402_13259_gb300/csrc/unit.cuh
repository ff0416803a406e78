// unit.cuh -- one (station, replication) update of the Euler step and the
// warp-level statistics reductions, shared by the library's kernels.
#pragma once

#include <cstdint>

#include "internal.h"
#include "sampling.cuh"

namespace eulernet {
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void latch(unsigned* err, unsigned bits) {
  if (bits) atomicOr(err, bits);
}

__device__ __forceinline__ BinomConst as_const(float4 v) { return BinomConst{v.x, v.y, v.z, v.w}; }

// Servers of station i during step tau (a staffing schedule, Sec. 2.1.2, or
// the constant m_i).
template <bool EXT = true>
__device__ __forceinline__ int32_t servers_at(const NetTables& t, const RunParams& p, int32_t i,
                                              uint32_t tau) {
  if (EXT && p.mtab) return __ldg(p.mtab + (int64_t)(tau - 1) * t.n + i);
  return __ldg(t.servers + i);
}

__device__ __forceinline__ int64_t gather_in(const NetTables& t, int32_t i, const int32_t* redge,
                                             int64_t stride, int64_t col) {
  int64_t s = 0;
  const int32_t k1 = __ldg(t.in_ptr + i + 1);
  for (int32_t k = __ldg(t.in_ptr + i); k < k1; ++k)
    s += redge[(int64_t)__ldg(t.in_edge + k) * stride + col];
  return s;
}

// Sum `v` over aligned segments of `w` lanes (w a power of two <= 32); the
// segment total ends up in every lane of the segment.
__device__ __forceinline__ unsigned seg_sum32(unsigned v, int w) {
  if (w == 32) return __reduce_add_sync(kFull, v);
  for (int off = w >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

__device__ __forceinline__ long long seg_sum64(long long v, int w) {
  for (int off = w >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Reduce NV per-unit values over the replication segment and add them to
// dst[0..NV) by the segment leader.  `fits` must be warp-uniform-safe: it is
// combined with __all_sync here.  mode 0: plain add (exclusive owner), 1:
// shared/global atomic add.
template <int NV>
__device__ __forceinline__ void reduce_to(long long* dst, const int32_t (&v)[NV], bool lead,
                                          int w, bool atomic) {
  int32_t vmax = 0;
#pragma unroll
  for (int s = 0; s < NV; ++s) vmax = v[s] > vmax ? v[s] : vmax;
  const bool small = __all_sync(kFull, vmax < (1 << 27));
  long long tot[NV];
  if (small) {
#pragma unroll
    for (int s = 0; s < NV; ++s) tot[s] = (long long)seg_sum32((unsigned)v[s], w);
  } else {
#pragma unroll
    for (int s = 0; s < NV; ++s) tot[s] = seg_sum64((long long)v[s], w);
  }
  if (lead) {
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      if (atomic)
        atomicAdd(reinterpret_cast<unsigned long long*>(dst + s), (unsigned long long)tot[s]);
      else
        dst[s] += tot[s];
    }
  }
}

// ---- one unit ----------------------------------------------------------------

struct UnitOut {
  int32_t N, D, X, A;
  int32_t x;   // input count of the departure draw
  float smu;   // score term of the departure in mu_i (GRAD only)
  float garr;  // A/Lambda - 1 of an external-arrival draw, NaN if none (GRAD only)
};

// Departure then routing from input count y (Algorithm 1, then the Sec. 2.2
// multinomial as sequential conditional binomials), from the unit's service
// stream (Algorithm 1's Erlang time from its own stream, see
// departure_branch).  One binomial call site serves the departure and every
// routing edge, so lanes that took different branches of Algorithm 1 execute
// the binomial together.
// EXT: the run may use a staffing schedule or the Eq. (1)/(2) samplers.
template <bool GRAD, bool EXT>
__device__ __forceinline__ void serve_and_route(const NetTables& t, const RunParams& p, int32_t i,
                                                uint32_t tau, uint32_t rep, int32_t y,
                                                int32_t* redge, int64_t stride, int64_t col,
                                                SamplerCtx& cx, int32_t& D, int32_t& X, float& smu,
                                                const uint32_t* rk = nullptr) {
  PhiloxStream svc;
  svc.init(p.key0, p.key1, 1u, (uint32_t)i, tau, rep, rk);
  const int32_t m = servers_at<EXT>(t, p, i, tau);
  // Block 0 of the stream now, while the warp's lanes still run together
  // (the first draw would compute the same block inside a divergent branch).
  svc.refill();
  const int32_t e0 = __ldg(t.row_ptr + i);
  const int32_t deg = __ldg(t.row_ptr + i + 1) - e0;
  int32_t rem = 0;
  int32_t j0 = -1;
  D = 0;
  BinomialArgs dep;
  if (EXT && (p.dep_mode == 1 || (p.dep_mode == 2 && y > m))) {
    // Eq. (1) (Eq. (2) for x > m): D = min(x, Poisson(min(x, m) mu h))
    const int32_t b = y < m ? y : m;
    const int32_t S = poisson((float)b * __ldg(p.muh + i), svc, cx);
    D = S < y ? S : y;
    rem = D;
    j0 = 0;
  } else {
    dep = departure_branch(y, m, __ldg(t.mu + i), p.h, as_const(__ldg(p.p0 + i)), svc, cx);
  }
  for (int32_t j = j0; j < deg; ++j) {
    const int32_t nb = j < 0 ? dep.n : rem;
    const BinomConst bc = j < 0 ? dep.c : as_const(__ldg(t.qc + e0 + j));
    const int32_t v = binomial_c(nb, bc, svc, cx);  // Bin(0, .) draws nothing
    if (j < 0) {
      D = dep.base + v;
      rem = D;
      if (GRAD) {
        // d/dmu_i of the log-probability of this departure (float32):
        //   x <= m : Bin(x, p0(mu)), dp0/dmu = h(1 - p0)        -> h (k/p0 - x)
        //   x >  m : Erlang(x - m, m mu) density at T            -> (x - m)/mu - m T
        //            plus, if T <= h, Bin(m, p(mu)), dp/dmu = (h - T)(1 - p) -> (h - T)(k/p - m)
        if (dep.branch == 0) {
          smu = p.h * ((v > 0 ? (float)v / __ldg(p.p0f + i) : 0.0f) - (float)y);
        } else {
          const float mu = __ldg(t.mu + i);
          const float te = (float)(y - m) / mu - (float)m * dep.T;
          smu = dep.branch == 1 ? te : te + (p.h - dep.T) * ((v > 0 ? (float)v / dep.p : 0.0f) - (float)m);
        }
      }
    } else {
      redge[(int64_t)(e0 + j) * stride + col] = v;
      rem = rem - v;
    }
  }
  X = rem;
}

// One unit of either scheme at station i.  The external-arrival draw comes
// first: it uses its own stream, so its position does not change any draw.
//   FULL = true  (forward, Algorithm 3): x = N_{tau-1} + A^ex + A^in, N_tau = x - D.
//   FULL = false (backward, Algorithm 2, first phase): x = N_{tau-1};
//                stores N_{tau-1} - D + A^ex, the gather adds A^in later.
template <bool FULL, bool GRAD = false, bool EXT = true>
__device__ __forceinline__ UnitOut unit_update(const NetTables& t, const RunParams& p, int32_t i,
                                               uint32_t tau, uint32_t rep, const float* lam_t,
                                               int32_t* nstate, int32_t* redge, int64_t stride,
                                               int64_t col, SamplerCtx& cx, const uint32_t* rk = nullptr) {
  UnitOut o;
  o.A = 0;
  o.smu = 0.0f;
  o.garr = __int_as_float(0x7fc00000);
  const int32_t ec = __ldg(t.ex_col + i);
  if (ec >= 0) {
    PhiloxStream arr;
    arr.init(p.key0, p.key1, 0u, (uint32_t)i, tau, rep, rk);
    arr.refill();  // every Poisson draw takes at least one word
    const float lam = __ldg(lam_t + ec);
    o.A = poisson(lam, arr, cx);
    if (GRAD && lam > 0.0f) o.garr = (float)o.A / lam - 1.0f;  // d log Poisson / d Lambda * Lambda / Lambda
  }
  const int32_t n_prev = nstate[(int64_t)i * stride + col];
  long long x = n_prev;
  if (FULL) {
    x += (long long)o.A + gather_in(t, i, redge, stride, col);
    if (x > kStateLimit) {
      cx.err |= kErrOverflow;
      x = kStateLimit;
    }
  }
  serve_and_route<GRAD, EXT>(t, p, i, tau, rep, (int32_t)x, redge, stride, col, cx, o.D, o.X, o.smu, rk);
  o.x = (int32_t)x;
  if (FULL) {
    o.N = (int32_t)x - o.D;
    nstate[(int64_t)i * stride + col] = o.N;
  } else {
    long long part = (long long)n_prev - o.D + o.A;
    if (part > 0x7fffffffLL) part = 0x7fffffffLL;
    nstate[(int64_t)i * stride + col] = (int32_t)part;
    o.N = 0;
  }
  return o;
}

// Backward second phase: N_tau = (N_{tau-1} - D + A^ex) + A^in.
__device__ __forceinline__ int32_t backward_gather(const NetTables& t, int32_t i, int32_t* nstate,
                                                   const int32_t* redge, int64_t stride,
                                                   int64_t col, unsigned& err) {
  long long nn = (long long)nstate[(int64_t)i * stride + col] + gather_in(t, i, redge, stride, col);
  if (nn > kStateLimit) {
    err |= kErrOverflow;
    nn = kStateLimit;
  }
  nstate[(int64_t)i * stride + col] = (int32_t)nn;
  return (int32_t)nn;
}

// 1/k for k < 64 (entry 0 unused), each the correctly rounded quotient: the
// compiler folds the constant divisions.
__device__ const float kRinvTable[64] = {
    0.0f, 1.0f / 1.0f, 1.0f / 2.0f, 1.0f / 3.0f, 1.0f / 4.0f, 1.0f / 5.0f, 1.0f / 6.0f, 1.0f / 7.0f,
    1.0f / 8.0f, 1.0f / 9.0f, 1.0f / 10.0f, 1.0f / 11.0f, 1.0f / 12.0f, 1.0f / 13.0f, 1.0f / 14.0f, 1.0f / 15.0f,
    1.0f / 16.0f, 1.0f / 17.0f, 1.0f / 18.0f, 1.0f / 19.0f, 1.0f / 20.0f, 1.0f / 21.0f, 1.0f / 22.0f, 1.0f / 23.0f,
    1.0f / 24.0f, 1.0f / 25.0f, 1.0f / 26.0f, 1.0f / 27.0f, 1.0f / 28.0f, 1.0f / 29.0f, 1.0f / 30.0f, 1.0f / 31.0f,
    1.0f / 32.0f, 1.0f / 33.0f, 1.0f / 34.0f, 1.0f / 35.0f, 1.0f / 36.0f, 1.0f / 37.0f, 1.0f / 38.0f, 1.0f / 39.0f,
    1.0f / 40.0f, 1.0f / 41.0f, 1.0f / 42.0f, 1.0f / 43.0f, 1.0f / 44.0f, 1.0f / 45.0f, 1.0f / 46.0f, 1.0f / 47.0f,
    1.0f / 48.0f, 1.0f / 49.0f, 1.0f / 50.0f, 1.0f / 51.0f, 1.0f / 52.0f, 1.0f / 53.0f, 1.0f / 54.0f, 1.0f / 55.0f,
    1.0f / 56.0f, 1.0f / 57.0f, 1.0f / 58.0f, 1.0f / 59.0f, 1.0f / 60.0f, 1.0f / 61.0f, 1.0f / 62.0f, 1.0f / 63.0f,
};

__device__ __forceinline__ void fill_rinv(float* rinv) {
  for (int k = threadIdx.x; k < 64; k += blockDim.x) rinv[k] = kRinvTable[k];
}

}  // namespace eulernet
