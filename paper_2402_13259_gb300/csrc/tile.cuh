// tile.cuh -- one tile of replications of the persistent shared-memory form:
// the whole time loop of Algorithm 2 (backward) or Algorithm 3 (forward) for
// Rt replications of one network, with the state in shared memory.  Shared by
// the library's persistent, batched and sojourn-time kernels.
#pragma once

#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "sampling.cuh"
#include "unit.cuh"

namespace eulernet {

// Per-tile extension points of tile_body; the plain kernels use this empty one.
//   unit(i, r, tau, o): after the unit update of station i, replication slot r
//   step_end(tau, ...): after the block barrier that ends step tau; an
//                       implementation that touches shared state must end
//                       with a block barrier of its own
//   tile_end(tile):     after the time loop, before the statistics epilogue
struct NoHook {
  __device__ __forceinline__ void unit(int32_t, int, int32_t, const UnitOut&) {}
  __device__ __forceinline__ void step_end(int32_t, int64_t, const int32_t*, const int32_t*) {}
  __device__ __forceinline__ void tile_end(int64_t) {}
};

// Per-station sums of a CTA into the stats buffer (integer atomics, so the
// result does not depend on the order).
__device__ __forceinline__ void flush_station_sums(const NetTables& t, const RunParams& p,
                                                   const long long* sacc) {
  const int32_t n = t.n;
  int64_t* st_nk = p.stats + 5 * (int64_t)n + 4 * p.R;
  for (int64_t k = threadIdx.x; k < 6 * (int64_t)n; k += blockDim.x) {
    const int64_t i = k / 6, s = k % 6;
    const long long v = sacc[k];
    if (v == 0) continue;
    unsigned long long* dst =
        reinterpret_cast<unsigned long long*>(s < 5 ? p.stats + i * 5 + s : st_nk + i);
    atomicAdd(dst, (unsigned long long)v);
  }
}

// ---- persistent shared-memory form -------------------------------------------

// Pointers into a CTA's working area for one tile of `Rt` replications of one
// network.  sacc may live in shared memory or, for networks whose per-station
// accumulators do not fit, in a global scratch slot owned by the CTA.
struct TileSmem {
  float* rinv;      // [64] 1/k
  long long* sacc;  // [n][6] per-station sums (owned by this CTA)
  long long* racc;  // [Rt][4] per-replication sums of the tile
  int32_t* Ns;      // [n][Rt] state
  int32_t* Rs;      // [E][Rt] routed counts
  int* claim;       // [2] dynamic station claims per phase parity
  double* mu_acc;   // GRAD: [n][Rt] score sums in mu_i
  double* th_acc;   // GRAD: [n_ex][Rt][3] score sums in (a, b, phase) per external station
};

// Score terms of one unit into the tile's accumulators (GRAD kernels).
__device__ __forceinline__ void add_scores(const NetTables& t, const RunParams& p, const TileSmem& sm,
                                           int32_t i, int32_t tau, int r, int Rt, const UnitOut& o) {
  sm.mu_acc[(int64_t)i * Rt + r] += (double)o.smu;
  if (!isnan(o.garr)) {
    const int32_t ec = __ldg(t.ex_col + i);
    const float* dl = p.dlam + ((int64_t)(tau - 1) * t.n_ex + ec) * 3;
    double* th = sm.th_acc + ((int64_t)ec * Rt + r) * 3;
    th[0] += (double)(o.garr * __ldg(dl + 0));
    th[1] += (double)(o.garr * __ldg(dl + 1));
    th[2] += (double)(o.garr * __ldg(dl + 2));
  }
}

// One tile: the whole time loop for replications tile*Rt ... of network t.
// Adds per-station sums (and N_K) into sm.sacc and writes the tile's
// per-replication sums to p.stats.  Ends with a block barrier.
// rk: the Philox round keys in the kernel's parameter space, or nullptr.
//
// Without a hook the loop runs in slots, one block barrier each, with the
// routed counts in t.ring slots of sm.Rs ([ring][E][Rt]):
//   backward (Algorithm 2), slot tau = 1 .. K+1: every station gathers its
//     routed counts of step tau-1 (ring slot (tau-1) % 2) and completes
//     N_{tau-1}, then draws step tau from it into ring slot tau % 2 -- one
//     barrier per step instead of two;
//   forward (Algorithm 3), slot tau = 1 .. K+L-1: the station at level l
//     runs step tau - l, so its predecessors ran that step and it ran its own
//     previous step in earlier slots; routed counts of step s stay in ring
//     slot s % ring until their consumer has read them -- one barrier per
//     slot instead of one per level and step.
// Every station's steps still run in order, so the state, the integer sums
// and each per-(station, replication) score sum are those of the step loop.
// With a hook (which sees the whole network after each step) the loop runs
// step by step: a barrier after each phase (backward) or level (forward),
// routed counts in one slot.
template <int SCHEME, bool GRAD = false, bool EXT = true, class Hook = NoHook>
__device__ __forceinline__ void tile_body(const NetTables& t, const RunParams& p, int64_t tile,
                                          const TileSmem& sm, SamplerCtx& cx, Hook& hook,
                                          const uint32_t* rk = nullptr) {
  const int32_t n = t.n;
  const int Rt = p.tile_reps;
  long long* sacc = sm.sacc;
  long long* racc = sm.racc;
  int32_t* Ns = sm.Ns;
  int32_t* Rs = sm.Rs;
  int* claim = sm.claim;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int r = tid % Rt;
  const int g0 = tid / Rt;
  const int G = nthr / Rt;
  const int lane = tid & 31;
  const int w = Rt < 32 ? Rt : 32;
  const int gwarp = (tid & ~31) / Rt;  // group of lane 0 of this warp
  const bool lead = (lane & (w - 1)) == 0;
  const bool shared_station = Rt > 32;  // several warps per station -> atomics
  // With one warp per station-unit (Rt = 32) warps claim the stations of a
  // phase dynamically; claim[phase parity] counts the stations handed out.
  const bool dynamic = Rt == 32;
  int phase = 0;

    const int64_t rloc = tile * Rt + r;
    const bool rvalid = rloc < p.R;
    const uint32_t rep = (uint32_t)(p.rep_begin + rloc);
    for (int64_t k = tid; k < (int64_t)n * Rt; k += nthr)
      Ns[k] = t.N0 ? __ldg(t.N0 + k / Rt) : 0;
    for (int k = tid; k < 4 * Rt; k += nthr) racc[k] = 0;
    if (GRAD) {
      for (int64_t k = tid; k < (int64_t)n * Rt; k += nthr) sm.mu_acc[k] = 0.0;
      for (int64_t k = tid; k < 3 * (int64_t)t.n_ex * Rt; k += nthr) sm.th_acc[k] = 0.0;
    }
    if (tid < 2) claim[tid] = 0;
    phase = 0;
    long long q_r = 0, d_r = 0, x_r = 0, a_r = 0;
    __syncthreads();

    // next station slot of this warp in the current phase (m slots)
    auto next_slot = [&](int su0, int m) -> int {
      if (!dynamic) return su0 + G;
      int s = 0;
      if (lane == 0) s = atomicAdd(&claim[phase & 1], 1);
      return __shfl_sync(kFull, s, 0);
    };
    auto first_slot = [&]() -> int {
      if (!dynamic) return gwarp;
      if (tid == 0) claim[(phase + 1) & 1] = 0;  // counter of the next phase
      int s = 0;
      if (lane == 0) s = atomicAdd(&claim[phase & 1], 1);
      return __shfl_sync(kFull, s, 0);
    };

    constexpr bool kSlots = std::is_same<Hook, NoHook>::value;
    if constexpr (kSlots) {
      const int64_t ring_stride = (int64_t)t.E * Rt;
      if (SCHEME == 0) {
        for (int32_t slot = 1; slot <= p.K + 1; ++slot) {
          const int32_t* rprev = Rs + (int64_t)((slot - 1) & 1) * ring_stride;
          int32_t* rcur = Rs + (int64_t)(slot & 1) * ring_stride;
          const float* lam_t = p.lam + (int64_t)(slot <= p.K ? slot - 1 : 0) * t.n_ex;
          for (int su0 = first_slot(); su0 < n; su0 = next_slot(su0, n)) {
            const int su = su0 + (g0 - gwarp);
            const bool act = rvalid && su < n;
            int32_t v[5] = {0, 0, 0, 0, 0};
            if (act) {
              if (slot >= 2) {
                const int32_t nn = backward_gather(t, su, Ns, rprev, Rt, r, cx.err);
                const int32_t c = servers_at<EXT>(t, p, su, (uint32_t)(slot - 1));
                v[0] = nn;
                v[1] = nn < c ? nn : c;
                q_r += nn;
              }
              if (slot <= p.K) {
                const UnitOut o = unit_update<false, GRAD, EXT>(t, p, su, (uint32_t)slot, rep, lam_t, Ns, rcur, Rt, r, cx, rk);
                if (GRAD) add_scores(t, p, sm, su, slot, r, Rt, o);
                v[2] = o.D;
                v[3] = o.X;
                v[4] = o.A;
                d_r += o.D;
                x_r += o.X;
                a_r += o.A;
              }
            }
            reduce_to<5>(sacc + 6 * (int64_t)(su < n ? su : 0), v, lead && su < n, w, shared_station);
          }
          ++phase;
          __syncthreads();
        }
      } else {
        for (int32_t slot = 1; slot <= p.K + t.L - 1; ++slot) {
          for (int su0 = first_slot(); su0 < n; su0 = next_slot(su0, n)) {
            const int su = su0 + (g0 - gwarp);
            const int32_t i = su < n ? __ldg(t.lvl_station + su) : 0;
            const int32_t tau = su < n ? slot - __ldg(t.pos_level + su) : 0;
            const bool live = su < n && tau >= 1 && tau <= p.K;
            int32_t v[5] = {0, 0, 0, 0, 0};
            if (rvalid && live) {
              int32_t* redge = Rs + (int64_t)(tau % t.ring) * ring_stride;
              const float* lam_t = p.lam + (int64_t)(tau - 1) * t.n_ex;
              const UnitOut o = unit_update<true, GRAD, EXT>(t, p, i, (uint32_t)tau, rep, lam_t, Ns, redge, Rt, r, cx, rk);
              if (GRAD) add_scores(t, p, sm, i, tau, r, Rt, o);
              const int32_t c = servers_at<EXT>(t, p, i, (uint32_t)tau);
              v[0] = o.N;
              v[1] = o.N < c ? o.N : c;
              v[2] = o.D;
              v[3] = o.X;
              v[4] = o.A;
              q_r += o.N;
              d_r += o.D;
              x_r += o.X;
              a_r += o.A;
            }
            reduce_to<5>(sacc + 6 * (int64_t)i, v, lead && live, w, shared_station);
          }
          ++phase;
          __syncthreads();
        }
      }
    } else
    for (int32_t tau = 1; tau <= p.K; ++tau) {
      const float* lam_t = p.lam + (int64_t)(tau - 1) * t.n_ex;
      if (SCHEME == 0) {
        for (int su0 = first_slot(); su0 < n; su0 = next_slot(su0, n)) {
          const int su = su0 + (g0 - gwarp);
          const bool act = rvalid && su < n;
          int32_t v[3] = {0, 0, 0};
          if (act) {
            const UnitOut o = unit_update<false, GRAD, EXT>(t, p, su, (uint32_t)tau, rep, lam_t, Ns, Rs, Rt, r, cx, rk);
            if (GRAD) add_scores(t, p, sm, su, tau, r, Rt, o);
            hook.unit(su, r, tau, o);
            v[0] = o.D;
            v[1] = o.X;
            v[2] = o.A;
            d_r += o.D;
            x_r += o.X;
            a_r += o.A;
          }
          reduce_to<3>(sacc + 6 * (int64_t)(su < n ? su : 0) + 2, v, lead && su < n, w,
                       shared_station);
        }
        ++phase;
        __syncthreads();
        for (int su0 = first_slot(); su0 < n; su0 = next_slot(su0, n)) {
          const int su = su0 + (g0 - gwarp);
          const bool act = rvalid && su < n;
          int32_t v[2] = {0, 0};
          if (act) {
            const int32_t nn = backward_gather(t, su, Ns, Rs, Rt, r, cx.err);
            const int32_t c = servers_at<EXT>(t, p, su, (uint32_t)tau);
            v[0] = nn;
            v[1] = nn < c ? nn : c;
            q_r += nn;
          }
          reduce_to<2>(sacc + 6 * (int64_t)(su < n ? su : 0), v, lead && su < n, w, shared_station);
        }
        ++phase;
        __syncthreads();
      } else {
        for (int32_t j = 0; j < t.L; ++j) {
          const int32_t s0 = __ldg(t.lvl_ptr + j);
          const int32_t m = __ldg(t.lvl_ptr + j + 1) - s0;
          for (int su0 = first_slot(); su0 < m; su0 = next_slot(su0, m)) {
            const int su = su0 + (g0 - gwarp);
            const bool act = rvalid && su < m;
            const int32_t i = su < m ? __ldg(t.lvl_station + s0 + su) : 0;
            int32_t v[5] = {0, 0, 0, 0, 0};
            if (act) {
              const UnitOut o = unit_update<true, GRAD, EXT>(t, p, i, (uint32_t)tau, rep, lam_t, Ns, Rs, Rt, r, cx, rk);
              if (GRAD) add_scores(t, p, sm, i, tau, r, Rt, o);
              hook.unit(i, r, tau, o);
              const int32_t c = servers_at<EXT>(t, p, i, (uint32_t)tau);
              v[0] = o.N;
              v[1] = o.N < c ? o.N : c;
              v[2] = o.D;
              v[3] = o.X;
              v[4] = o.A;
              q_r += o.N;
              d_r += o.D;
              x_r += o.X;
              a_r += o.A;
            }
            reduce_to<5>(sacc + 6 * (int64_t)i, v, lead && su < m, w, shared_station);
          }
          ++phase;
          __syncthreads();
        }
      }
      hook.step_end(tau, tile, Ns, Rs);
    }

    // tile epilogue: per-replication sums and N_K
    if (rvalid) {
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * r + 0), (unsigned long long)q_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * r + 1), (unsigned long long)d_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * r + 2), (unsigned long long)x_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * r + 3), (unsigned long long)a_r);
    }
    for (int su0 = gwarp; su0 < n; su0 += G) {
      const int su = su0 + (g0 - gwarp);
      int32_t v[1] = {(rvalid && su < n) ? Ns[(int64_t)su * Rt + r] : 0};
      reduce_to<1>(sacc + 6 * (int64_t)(su < n ? su : 0) + 5, v, lead && su < n, w, shared_station);
    }
    __syncthreads();
    hook.tile_end(tile);
    int64_t* st_rep = p.stats + 5 * (int64_t)n;
    for (int k = tid; k < 4 * Rt; k += nthr) {
      const int64_t rr = tile * Rt + k / 4;
      if (rr < p.R) st_rep[rr * 4 + (k & 3)] = racc[k];
    }
    if (GRAD) {
      // S_r: mu_i sums, then (a, b, phase) summed over external stations in order
      const int64_t C = (int64_t)n + 3;
      for (int64_t k = tid; k < C * Rt; k += nthr) {
        const int rr = (int)(k % Rt);
        const int64_t c = k / Rt;
        const int64_t rg = tile * Rt + rr;
        if (rg >= p.R) continue;
        double v;
        if (c < n) {
          v = sm.mu_acc[c * Rt + rr];
        } else {
          v = 0.0;
          for (int32_t ec = 0; ec < t.n_ex; ++ec) v += sm.th_acc[((int64_t)ec * Rt + rr) * 3 + (c - n)];
        }
        p.scores[rg * C + c] = v;
      }
    }
    __syncthreads();
}

}  // namespace eulernet
