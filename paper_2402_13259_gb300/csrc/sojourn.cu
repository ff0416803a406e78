// sojourn.cu -- euler_net_sojourn: sojourn times of tagged customers (Sec. 6,
// Algorithm 4, with the conditional stay probability of Lemma 3), sampled
// while the Euler time loop runs.  This file holds the persistent
// shared-memory form; at scale the HBM form's per-step kernels (kernels.cu)
// advance the customers instead, with the same results.
//
// Algorithm 4 reads, for each step after the customer's entry, the values
// that step produced at the customer's station: the departure draw's input x
// and output D, the post-update count N and the routed counts R_e.  Instead
// of storing whole sample paths and replaying them, the persistent kernel
// keeps each tile's tagged customers in shared memory and advances them once
// per step, right after the step's last block barrier, from that step's
// values (kept for one step in shared memory).  The outputs are those of
// Algorithm 4 run over the stored paths, step for step.
//
// Tagged customer c of a tile (replication slot r = c % Rt, sample s = c / Rt)
// has a station, a state (position > 0 while waiting, 0 in service, -1 after
// leaving the network) and the steps accounted so far:
//   setup at station i after step tau: pos = max(N_tau,i, 1); wait if pos > m_i
//   waiting, step tau:  pos -= D_tau,i; in service from the next step once pos <= m_i
//   service, step tau:  stay with probability Lemma 3 (x_tau,i, D_tau,i, m_i):
//                       u < p_stay, u the first uniform of stream (seed,
//                       purpose 3, slot s, step tau, replication); otherwise
//                       the customer is departure k = floor(w D / 2^32) (w the
//                       stream's second word) of the step's D, which go to the
//                       row's edges in CSR order (R_e each) and then exit.
// m_i is the staffing of the step whose values are read.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "handle.h"
#include "internal.h"
#include "sampling.cuh"
#include "tile.cuh"
#include "unit.cuh"

namespace eulernet {
namespace {

struct SojournParams {
  const int32_t* col;  // [E] destination station of each edge
  int32_t* out;        // [R][S] sojourn in steps (> 0), or -(steps) if censored
  int32_t station;     // entry station i0
  int32_t tau0;        // entry step, 1 <= tau0 <= K
  int32_t S;           // tagged customers per replication
};

// b^k (k >= 0) by binary powering, multiplications in a fixed order.
__device__ __forceinline__ float pow_int(float b, int32_t k) {
  float r = 1.0f;
  while (k > 0) {
    if (k & 1) r = r * b;
    b = b * b;
    k >>= 1;
  }
  return r;
}

// Lemma 3: P(the tagged customer's service continues through the step | the
// step's departure draw had input x and output d, m servers); d > 0.
__device__ __forceinline__ float stay_probability(int32_t x, int32_t d, int32_t m) {
  if (x <= m) return (float)(x - d) / (float)x;
  const float q = (float)(m - 1) / (float)m;
  if (x <= m + d) return pow_int(q, x - m) * ((float)(x - d) / (float)m);
  return pow_int(q, d);
}

template <bool EXT>
struct SojournHook {
  const NetTables* t;
  const RunParams* p;
  SojournParams q;
  int32_t* xs;      // [n][Rt] departure input of the current step
  int32_t* ds;      // [n][Rt] departures of the current step
  int32_t* cst;     // [S][Rt] station of each tagged customer
  int32_t* cpos;    // [S][Rt] > 0 waiting position, 0 in service, -1 left
  int32_t* csteps;  // [S][Rt] steps accounted

  __device__ __forceinline__ void unit(int32_t i, int r, int32_t tau, const UnitOut& o) {
    if (tau > q.tau0) {
      const int64_t k = (int64_t)i * p->tile_reps + r;
      xs[k] = o.x;
      ds[k] = o.D;
    }
  }

  __device__ __forceinline__ void setup(int c, int r, int32_t i, int32_t tau, const int32_t* Ns) {
    int32_t pos = Ns[(int64_t)i * p->tile_reps + r];
    if (pos < 1) pos = 1;
    cst[c] = i;
    cpos[c] = pos > servers_at<EXT>(*t, *p, i, (uint32_t)tau) ? pos : 0;
  }

  __device__ __forceinline__ void step_end(int32_t tau, int64_t tile, const int32_t* Ns,
                                           const int32_t* Rs) {
    if (tau < q.tau0) return;  // uniform across the block
    const int Rt = p->tile_reps;
    const int SR = q.S * Rt;
    for (int c = threadIdx.x; c < SR; c += blockDim.x) {
      const int r = c % Rt;
      const int64_t rloc = tile * Rt + r;
      if (rloc >= p->R) continue;
      if (tau == q.tau0) {
        setup(c, r, q.station, tau, Ns);
        csteps[c] = 0;
        continue;
      }
      int32_t pos = cpos[c];
      if (pos < 0) continue;
      const int32_t i = cst[c];
      csteps[c] += 1;
      const int32_t m = servers_at<EXT>(*t, *p, i, (uint32_t)tau);
      const int64_t k = (int64_t)i * Rt + r;
      const int32_t d = ds[k];
      if (pos > 0) {  // waiting step
        pos -= d;
        cpos[c] = pos <= m ? 0 : pos;
        continue;
      }
      if (d <= 0) continue;  // no departure: p_stay = 1
      const float ps = stay_probability(xs[k], d, m);
      PhiloxStream cs;
      cs.init(p->key0, p->key1, 3u, (uint32_t)(c / Rt), (uint32_t)tau,
              (uint32_t)(p->rep_begin + rloc));
      const float u = cs.uniform();
      const uint32_t w = cs.next();
      if (u < ps) continue;
      uint32_t pick = __umulhi(w, (uint32_t)d);
      int32_t next = -1;
      const int32_t e1 = __ldg(t->row_ptr + i + 1);
      for (int32_t e = __ldg(t->row_ptr + i); e < e1; ++e) {
        const uint32_t v = (uint32_t)Rs[(int64_t)e * Rt + r];
        if (pick < v) {
          next = __ldg(q.col + e);
          break;
        }
        pick -= v;
      }
      if (next < 0) {
        cpos[c] = -1;
      } else {
        setup(c, r, next, tau, Ns);
      }
    }
    __syncthreads();
  }

  __device__ __forceinline__ void tile_end(int64_t tile) {
    const int Rt = p->tile_reps;
    for (int c = threadIdx.x; c < q.S * Rt; c += blockDim.x) {
      const int64_t rloc = tile * Rt + c % Rt;
      if (rloc >= p->R) continue;
      const int32_t st = csteps[c];
      q.out[rloc * q.S + c / Rt] = cpos[c] < 0 ? st : -st;
    }
  }
};

template <int SCHEME, bool EXT>
__global__ void __launch_bounds__(512, 2) sojourn_kernel(NetTables t, RunParams p, SojournParams q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int claim[2];
  const int32_t n = t.n;
  const int Rt = p.tile_reps;
  TileSmem sm;
  sm.rinv = reinterpret_cast<float*>(smem);
  sm.sacc = reinterpret_cast<long long*>(smem + 256);
  sm.racc = sm.sacc + 6 * (int64_t)n;
  sm.Ns = reinterpret_cast<int32_t*>(sm.racc + 4 * (int64_t)Rt);
  sm.Rs = sm.Ns + (int64_t)n * Rt;
  sm.claim = claim;
  sm.mu_acc = sm.th_acc = nullptr;
  SojournHook<EXT> hook;
  hook.t = &t;
  hook.p = &p;
  hook.q = q;
  hook.xs = sm.Rs + (int64_t)t.E * Rt;
  hook.ds = hook.xs + (int64_t)n * Rt;
  hook.cst = hook.ds + (int64_t)n * Rt;
  hook.cpos = hook.cst + (int64_t)q.S * Rt;
  hook.csteps = hook.cpos + (int64_t)q.S * Rt;
  const int tid = threadIdx.x, nthr = blockDim.x;
  fill_rinv(sm.rinv);
  for (int64_t k = tid; k < 6 * (int64_t)n; k += nthr) sm.sacc[k] = 0;
  SamplerCtx cx{sm.rinv, p.cap, 0u};
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x)
    tile_body<SCHEME, false, EXT>(t, p, tile, sm, cx, hook);
  flush_station_sums(t, p, sm.sacc);
  latch(p.err, cx.err);
}

const void* sojourn_fn(int scheme, bool ext) {
  if (scheme == 0) return ext ? (const void*)sojourn_kernel<0, true> : (const void*)sojourn_kernel<0, false>;
  return ext ? (const void*)sojourn_kernel<1, true> : (const void*)sojourn_kernel<1, false>;
}

int64_t sojourn_smem_bytes(int32_t n, int32_t E, int32_t Rt, int32_t S) {
  return persistent_smem_bytes(n, E, 1, Rt) + 8 * (int64_t)n * Rt + 12 * (int64_t)S * Rt;
}

int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  set_last_error(buf);
  return e == cudaErrorMemoryAllocation ? EULER_ERR_OOM : EULER_ERR_CUDA;
}

}  // namespace
}  // namespace eulernet

using namespace eulernet;

extern "C" int euler_net_sojourn(euler_net* h, int32_t scheme, double dt, double T, int64_t R,
                                 uint64_t seed, int64_t rep_begin, int32_t station, int64_t tau0,
                                 int32_t samples, int32_t* sojourn, int64_t* stats, void* stream) try {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  if (scheme != EULER_BACKWARD && scheme != EULER_FORWARD) return fail(EULER_ERR_ARG, "unknown scheme");
  if (!(dt > 0.0) || !(T > 0.0) || !std::isfinite(dt) || !std::isfinite(T))
    return fail(EULER_ERR_ARG, "dt and T must be finite and > 0");
  if (R < 0 || rep_begin < 0) return fail(EULER_ERR_ARG, "replications and rep_begin must be >= 0");
  if (rep_begin + R > (int64_t)1 << 32) return fail(EULER_ERR_TOO_LARGE, "replication index beyond 2^32");
  const int64_t K = euler_num_steps(dt, T);
  if (K >= (1 << 24)) return fail(EULER_ERR_TOO_LARGE, "too many steps (T/dt >= 2^24)");
  if (station < 0 || station >= h->n) return fail(EULER_ERR_ARG, "entry station out of range");
  if (tau0 < 1 || tau0 > K) return fail(EULER_ERR_ARG, "entry step must be in [1, K]");
  if (samples < 1 || samples > (1 << 16)) return fail(EULER_ERR_ARG, "samples must be in [1, 65536]");
  if (R > 0 && !sojourn) return fail(EULER_ERR_ARG, "sojourn output is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!h->d_col && h->E > 0) {
    e = cudaMalloc(&h->d_col, sizeof(int32_t) * (size_t)h->E);
    if (e != cudaSuccess) return cuda_fail(e, "edge table");
    e = cudaMemcpy(h->d_col, h->col.data(), sizeof(int32_t) * (size_t)h->E, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "edge table upload");
    h->h2d_bytes += (int64_t)sizeof(int32_t) * h->E;
  }
  const size_t len = (size_t)euler_stats_len(h->n, R);
  if (!stats) {
    if (len > h->sstats_cap) {
      cudaFree(h->d_sstats);
      h->d_sstats = nullptr;
      h->sstats_cap = 0;
      e = cudaMalloc(&h->d_sstats, sizeof(int64_t) * len);
      if (e != cudaSuccess) return cuda_fail(e, "statistics scratch");
      h->sstats_cap = len;
    }
    stats = h->d_sstats;
  }
  int rc = prepare_step_tables(h, dt, T, s);
  if (rc) return rc;
  e = cudaMemsetAsync(stats, 0, sizeof(int64_t) * len, s);
  if (e != cudaSuccess) return cuda_fail(e, "statistics clear");
  if (R == 0) return EULER_OK;
  RunParams p;
  std::memset(&p, 0, sizeof p);
  p.p0 = h->d_p0;
  p.lam = h->d_lam;
  p.h = (float)dt;
  p.K = (int32_t)K;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.R = R;
  p.rep_begin = rep_begin;
  p.scheme = scheme;
  p.cap = h->opt[EULER_OPT_SAMPLER_CAP] > 0 ? (int32_t)h->opt[EULER_OPT_SAMPLER_CAP] : 1000;
  p.stats = stats;
  p.err = h->d_err;
  p.wait_limit = (int64_t)1 << 25;
  p.muh = h->d_muh;
  p.dep_mode = h->dep_mode();
  p.mtab = h->mtab();
  // At scale the HBM form, as for euler_net_simulate: the customers' state
  // lives in global memory and the warp of a customer's station advances it.
  const int forced = (int)h->opt[EULER_OPT_FORM];
  if (forced == 2 || (forced <= 0 && (int64_t)h->n * R >= kHbmMinUnitsPerStep)) {
    const int64_t ld = (R + 3) / 4 * 4;
    const size_t need = (size_t)samples * (size_t)ld;
    if (need > h->cust_cap) {
      cudaFree(h->d_cloc);
      cudaFree(h->d_cpos);
      cudaFree(h->d_csteps);
      h->d_cloc = nullptr;
      h->d_cpos = h->d_csteps = nullptr;
      h->cust_cap = 0;
      e = cudaMalloc(&h->d_cloc, sizeof(unsigned long long) * need);
      if (e == cudaSuccess) e = cudaMalloc(&h->d_cpos, sizeof(int32_t) * need);
      if (e == cudaSuccess) e = cudaMalloc(&h->d_csteps, sizeof(int32_t) * need);
      if (e != cudaSuccess) return cuda_fail(e, "sojourn customer state");
      h->cust_cap = need;
    }
    const int block = h->opt[EULER_OPT_BLOCK] > 0 ? (int)h->opt[EULER_OPT_BLOCK] : kHbmBlock;
    if (block % 32 || block > 256) return fail(EULER_ERR_ARG, "HBM-form block must be a multiple of 32 <= 256");
    p.tile_reps = 32;
    p.num_tiles = (R + 31) / 32;
    HbmExtra x;
    x.mode = kHbmSojourn;
    x.cloc = h->d_cloc;
    x.cpos = h->d_cpos;
    x.csteps = h->d_csteps;
    x.col = h->d_col;
    x.S = samples;
    x.station = station;
    x.tau0 = (int32_t)tau0;
    x.out = sojourn;
    return run_hbm_form(h, h->tables(), p, block, s, x);
  }
  // tile: the largest power of two <= 32 whose state and customers fit
  int Rt = 32;
  int64_t smem = 0;
  for (; Rt >= 1; Rt /= 2) {
    smem = sojourn_smem_bytes(h->n, h->E, Rt, samples);
    if (smem <= h->smem_optin) break;
  }
  if (Rt < 1) return fail(EULER_ERR_TOO_LARGE, "sojourn tile does not fit in shared memory");
  const int64_t m_max = scheme == EULER_BACKWARD ? h->n : h->max_level;
  const int quantum = Rt >= 32 ? 1 : 32 / Rt;
  const int64_t gmax = std::max<int64_t>(512 / Rt, 1);
  const int64_t iters = (m_max + gmax - 1) / gmax;
  int64_t G = (m_max + iters - 1) / iters;
  G = (G + quantum - 1) / quantum * quantum;
  if (G * Rt > 512) G = 512 / Rt;
  const int block = (int)std::max<int64_t>(G * Rt, 32);
  p.tile_reps = Rt;
  p.num_tiles = (R + Rt - 1) / Rt;
  SojournParams q;
  q.col = h->d_col;
  q.out = sojourn;
  q.station = station;
  q.tau0 = (int32_t)tau0;
  q.S = samples;
  const bool ext = p.mtab != nullptr || p.dep_mode != 0;
  const void* fn = sojourn_fn(scheme, ext);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "sojourn kernel attributes");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "sojourn occupancy query");
  if (per_sm < 1) return fail(EULER_ERR_TOO_LARGE, "sojourn kernel cannot be resident");
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * h->sm_count, p.num_tiles));
  NetTables t = h->tables();
  void* args[] = {&t, &p, &q};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(block), args, (size_t)smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "sojourn kernel launch");
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}
