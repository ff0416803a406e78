// hbm_step.cuh -- the HBM form's per-step kernel: one launch per step (or
// skewed slot) over all stations, state in global memory, one warp per
// (station, 32 replications), no block barrier.  The benchmark's kernel.
#pragma once

#include <cstdint>

#include "internal.h"
#include "sampling.cuh"
#include "unit.cuh"

namespace eulernet {
namespace {

// ---- HBM-state form -------------------------------------------------------------

constexpr int kHbmTile = 32;  // replications per CTA column of the HBM form

#ifndef EN_HBM_MIN_BLOCKS
#define EN_HBM_MIN_BLOCKS 5  // resident 256-thread CTAs per SM the register budget targets
#endif

// Units of one phase over stations lvl_station[s0 .. s0+m) (phases 2, 3) or
// 0 .. m (phases 0, 1, 4), at device counter + koff.  Grid: x over
// replication tiles of 32, y over station chunks; one warp per station and
// tile.
//   0: backward departures / routing / arrivals of step tau (Algorithm 2)
//   1: backward gather / update of step tau
//   4: backward, fused slot tau (1 .. K+1): the gather / update of step
//      tau - 1 (routed counts of the previous launch, ring slot (tau-1) % 2),
//      then the departures / routing / arrivals of step tau from that N_{tau-1}
//      (ring slot tau % 2): one launch per step instead of two
//   2: forward units of one level of step tau (Algorithm 3)
//   3: forward, skewed slot tau: station i at level l runs step tau - l.  Its
//      predecessors (lower levels) ran that step in earlier slots and its own
//      previous step in the previous slot, so every dependency of Algorithm 3
//      is met with one launch per slot for all stations; routed counts of
//      step s live in ring slot s % depth until their consumer has read them.
// Warps never wait for one another: each keeps its own 1/k table, adds its
// station sums with one warp reduction and its per-replication sums with one
// atomic per value, so a warp whose station drew cheap samples leaves at once.
// Score terms of one unit into the HBM form's per-(station, replication)
// sums: each cell belongs to one lane, so the float64 sums run in step order.
__device__ __forceinline__ void hbm_add_scores(const NetTables& t, const RunParams& p,
                                               const HbmState& hs, int32_t i, int32_t tau,
                                               int64_t rloc, const UnitOut& o) {
  hs.mu_acc[(int64_t)i * hs.ld + rloc] += (double)o.smu;
  if (!isnan(o.garr)) {
    const int32_t ec = __ldg(t.ex_col + i);
    const float* dl = p.dlam + ((int64_t)(tau - 1) * t.n_ex + ec) * 3;
    double* th = hs.th_acc + (int64_t)ec * 3 * hs.ld + rloc;
    th[0] += (double)(o.garr * __ldg(dl + 0));
    th[hs.ld] += (double)(o.garr * __ldg(dl + 1));
    th[2 * hs.ld] += (double)(o.garr * __ldg(dl + 2));
  }
}

// ---- sojourn times in the HBM form (Sec. 6, Algorithm 4, Lemma 3) ----------
//
// Tagged customer c of replication r has a packed word station << 32 | due
// step << 1 | setup pending, a place (> 0 waiting, 0 in service) and a step
// count.  The warp of the customer's station acts on it when it processes the
// due step: a setup reads N of that step (the place is max(N, 1), waiting if
// above m); a waiting step subtracts the step's departures; a service step
// keeps the customer with Lemma 3's probability given the step's departure
// input x and departures d, else sends it along the step's routed counts to
// the next station (setup pending there for the same step) or out.  Another
// station's warp may read the word while it is rewritten in the same launch:
// it then sees either a different station or a due step it is not
// processing, so the 64-bit word is read and written whole.
constexpr unsigned long long kSojDone = 0xFFFFFFFFull << 32;

__device__ __forceinline__ unsigned long long soj_pack(int32_t station, int32_t due, bool setup) {
  return ((unsigned long long)(uint32_t)station << 32) | ((unsigned long long)(uint32_t)due << 1) |
         (setup ? 1ull : 0ull);
}

// b^k (k >= 0) by binary powering, multiplications in a fixed order.
__device__ __forceinline__ float soj_pow_int(float b, int32_t k) {
  float r = 1.0f;
  while (k > 0) {
    if (k & 1) r = r * b;
    b = b * b;
    k >>= 1;
  }
  return r;
}

// Lemma 3: P(the tagged customer's service continues through the step | the
// step's departure draw had input x and output d > 0, m servers).
__device__ __forceinline__ float soj_stay(int32_t x, int32_t d, int32_t m) {
  if (x <= m) return (float)(x - d) / (float)x;
  const float q = (float)(m - 1) / (float)m;
  if (x <= m + d) return soj_pow_int(q, x - m) * ((float)(x - d) / (float)m);
  return soj_pow_int(q, d);
}

// Setup of customer word *lp at station i after step tau (N = N_tau,i).
template <bool EXT>
__device__ __forceinline__ void soj_setup(const NetTables& t, const RunParams& p, const HbmState& hs,
                                          int64_t ci, int32_t i, int32_t tau, int32_t N) {
  const int32_t pos = N < 1 ? 1 : N;
  hs.cpos[ci] = pos > servers_at<EXT>(t, p, i, (uint32_t)tau) ? pos : 0;
  hs.cloc[ci] = soj_pack(i, tau + 1, false);
}

// Waiting or service step tau of customer ci at station i (x, d: the step's
// departure input and output; redge: its routed counts).
template <bool EXT>
__device__ __forceinline__ void soj_step(const NetTables& t, const RunParams& p, const HbmState& hs,
                                         int64_t ci, int32_t c, int32_t i, int32_t tau, uint32_t rep,
                                         int32_t x, int32_t d, const int32_t* redge, int64_t rloc) {
  hs.csteps[ci] += 1;
  const int32_t m = servers_at<EXT>(t, p, i, (uint32_t)tau);
  int32_t pos = hs.cpos[ci];
  if (pos > 0) {  // waiting step
    pos -= d;
    hs.cpos[ci] = pos <= m ? 0 : pos;
    hs.cloc[ci] = soj_pack(i, tau + 1, false);
    return;
  }
  if (d > 0) {
    const float ps = soj_stay(x, d, m);
    PhiloxStream cs;
    cs.init(p.key0, p.key1, 3u, (uint32_t)c, (uint32_t)tau, rep, hs.rk);
    const float u = cs.uniform();
    const uint32_t w = cs.next();
    if (!(u < ps)) {
      uint32_t pick = __umulhi(w, (uint32_t)d);
      const int32_t e1 = __ldg(t.row_ptr + i + 1);
      for (int32_t e = __ldg(t.row_ptr + i); e < e1; ++e) {
        const uint32_t v = (uint32_t)redge[(int64_t)e * hs.ld + rloc];
        if (pick < v) {
          hs.cloc[ci] = soj_pack(__ldg(hs.col + e), tau, true);
          return;
        }
        pick -= v;
      }
      hs.cloc[ci] = kSojDone;
      return;
    }
  }
  hs.cloc[ci] = soj_pack(i, tau + 1, false);  // still in service
}

template <int PHASE, bool EXT = true, bool GRAD = false, bool SOJ = false>
__global__ void __launch_bounds__(256, EN_HBM_MIN_BLOCKS) hbm_phase_kernel(NetTables t, RunParams p,
                                                           const __grid_constant__ HbmState hs,
                                                           int32_t s0, int32_t m, int32_t koff) {
  constexpr int phase = PHASE;
  __shared__ float rinv_s[8 * 64];
  // Let the next slot's CTAs be scheduled as this grid's CTAs finish; they
  // wait (below) for this grid's completion before reading any state.  In a
  // launch without programmatic serialisation both are no-ops.
  asm volatile("griddepcontrol.launch_dependents;");
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rinv = rinv_s + 64 * wib;
  for (int k = lane; k < 64; k += 32) rinv[k] = kRinvTable[k];
  __syncwarp();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int32_t slot = *hs.tau + koff;
  if (slot > (phase == 3 ? p.K + t.L - 1 : phase == 4 ? p.K + 1 : p.K)) return;  // uniform
  const int64_t rloc = (int64_t)blockIdx.x * kHbmTile + lane;
  const bool rok = rloc < p.R;
  const uint32_t rep = (uint32_t)(p.rep_begin + rloc);
  const int su = blockIdx.y * (blockDim.x >> 5) + wib;
  if (su >= m) return;  // uniform across the warp; no block barrier follows
  const bool lead = lane == 0;
  SamplerCtx cx{rinv, p.cap, 0u};
  int32_t part[4] = {0, 0, 0, 0};  // Q, D, X, A of this lane's replication
  {
    const int32_t i = phase == 2 || phase == 3 ? __ldg(t.lvl_station + s0 + su) : su;
    int32_t tau = slot;
    bool live = true;  // this station has a step in this slot
    int32_t* redge = hs.Redge;
    if (phase == 3) {
      tau = slot - __ldg(hs.pos_level + s0 + su);
      live = tau > p.tau0 && tau <= p.K;
      if (!live) return;  // uniform across the warp
      redge = hs.Redge + (int64_t)(tau % hs.depth) * t.E * hs.ld;
    }
    const bool act = rok && live;
    const float* lam_t = p.lam + (int64_t)(tau <= p.K ? tau - 1 : 0) * t.n_ex;
    long long* st = reinterpret_cast<long long*>(p.stats + 5 * (int64_t)i);
    if constexpr (phase == 0) {  // backward departures / routing / arrivals
      int32_t v[3] = {0, 0, 0};
      if (act) {
        const UnitOut o = unit_update<false, false, EXT>(t, p, i, (uint32_t)tau, rep, lam_t, hs.N, redge, hs.ld, rloc, cx, hs.rk);
        v[0] = o.D; v[1] = o.X; v[2] = o.A;
        part[1] += o.D; part[2] += o.X; part[3] += o.A;
      }
      reduce_to<3>(st + 2, v, lead, 32, true);
    } else if constexpr (phase == 1) {  // backward gather / update
      int32_t v[2] = {0, 0};
      if (act) {
        const int32_t nn = backward_gather(t, i, hs.N, redge, hs.ld, rloc, cx.err);
        const int32_t c = servers_at<EXT>(t, p, i, (uint32_t)tau);
        v[0] = nn; v[1] = nn < c ? nn : c;
        part[0] += nn;
      }
      reduce_to<2>(st, v, lead, 32, true);
    } else if constexpr (phase == 4) {  // backward, fused: gather tau - 1, then draw tau
      int32_t v[5] = {0, 0, 0, 0, 0};
      if (act) {
        if (slot >= p.tau0 + 2) {
          const int32_t* rprev = hs.Redge + (int64_t)((slot - 1) & 1) * t.E * hs.ld;
          const int32_t nn = backward_gather(t, i, hs.N, rprev, hs.ld, rloc, cx.err);
          const int32_t c = servers_at<EXT>(t, p, i, (uint32_t)(slot - 1));
          v[0] = nn; v[1] = nn < c ? nn : c;
          part[0] += nn;
        }
        if (slot <= p.K) {
          int32_t* rcur = hs.Redge + (int64_t)(slot & 1) * t.E * hs.ld;
          const UnitOut o = unit_update<false, GRAD, EXT>(t, p, i, (uint32_t)slot, rep, lam_t, hs.N, rcur, hs.ld, rloc, cx, hs.rk);
          if (GRAD) hbm_add_scores(t, p, hs, i, slot, rloc, o);
          v[2] = o.D; v[3] = o.X; v[4] = o.A;
          part[1] += o.D; part[2] += o.X; part[3] += o.A;
          if (SOJ) {
            // customers due here: setups of step slot-1 (N = v[0]), then the
            // waiting / service step slot (x = N_{slot-1}, d = D)
            for (int32_t c = 0; c < hs.S; ++c) {
              const int64_t ci = (int64_t)c * hs.ld + rloc;
              unsigned long long w = hs.cloc[ci];
              if ((uint32_t)(w >> 32) != (uint32_t)i) continue;
              if ((w & 1ull) && (int32_t)((uint32_t)w >> 1) == slot - 1) {
                soj_setup<EXT>(t, p, hs, ci, i, slot - 1, v[0]);
                w = hs.cloc[ci];
              }
              if (!(w & 1ull) && (int32_t)((uint32_t)w >> 1) == slot)
                soj_step<EXT>(t, p, hs, ci, c, i, slot, rep, o.x, o.D, rcur, rloc);
            }
          }
        } else if (SOJ && slot >= p.tau0 + 2) {  // slot K+1: the last setups only
          for (int32_t c = 0; c < hs.S; ++c) {
            const int64_t ci = (int64_t)c * hs.ld + rloc;
            const unsigned long long w = hs.cloc[ci];
            if ((uint32_t)(w >> 32) == (uint32_t)i && (w & 1ull) && (int32_t)((uint32_t)w >> 1) == slot - 1)
              soj_setup<EXT>(t, p, hs, ci, i, slot - 1, v[0]);
          }
        }
      }
      reduce_to<5>(st, v, lead, 32, true);
    } else {  // forward: one level (2) or a skewed slot (3)
      int32_t v[5] = {0, 0, 0, 0, 0};
      if (act) {
        const UnitOut o = unit_update<true, GRAD, EXT>(t, p, i, (uint32_t)tau, rep, lam_t, hs.N, redge, hs.ld, rloc, cx, hs.rk);
        if (GRAD) hbm_add_scores(t, p, hs, i, tau, rloc, o);
        if (SOJ) {  // customers due here at step tau: a waiting / service step, or a setup
          for (int32_t c = 0; c < hs.S; ++c) {
            const int64_t ci = (int64_t)c * hs.ld + rloc;
            const unsigned long long w = hs.cloc[ci];
            if ((uint32_t)(w >> 32) != (uint32_t)i || (int32_t)((uint32_t)w >> 1) != tau) continue;
            if (w & 1ull)
              soj_setup<EXT>(t, p, hs, ci, i, tau, o.N);
            else
              soj_step<EXT>(t, p, hs, ci, c, i, tau, rep, o.x, o.D, redge, rloc);
          }
        }
        const int32_t c = servers_at<EXT>(t, p, i, (uint32_t)tau);
        v[0] = o.N; v[1] = o.N < c ? o.N : c; v[2] = o.D; v[3] = o.X; v[4] = o.A;
        part[0] += o.N; part[1] += o.D; part[2] += o.X; part[3] += o.A;
      }
      reduce_to<5>(st, v, lead, 32, true);
    }
  }
  if (rok) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (part[s])
        atomicAdd(reinterpret_cast<unsigned long long*>(hs.racc + rloc * 4 + s),
                  (unsigned long long)(long long)part[s]);
  }
  latch(p.err, cx.err);
}

}  // namespace
}  // namespace eulernet
