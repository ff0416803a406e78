// pipeline.cu -- the Euler step with the stations of a replication tile split
// over warps that run their own time loops, synchronised only with the warps
// they exchange routed customers with (no block-wide barriers in the loop).
//
// A CTA owns a tile of 32 replications (lane = replication).  The stations,
// in level order (longest path from a source, so every routing edge goes to a
// later position), are cut into W contiguous slices, one per warp.  Routed
// counts R_e live in two shared-memory buffers selected by step parity.  Per
// warp two progress counters in shared memory: ph1[w] = last step whose R_e
// the warp has written, done[w] = last step it has finished.
//   forward (Algorithm 3): before step tau a warp waits for its producer warps
//     (owners of its stations' predecessors) to reach ph1 >= tau -- their
//     routed counts of this step -- and for its consumer warps to reach
//     done >= tau - 2, so the buffer it is about to overwrite has been read.
//     Within the warp stations run in level order.
//   backward (Algorithm 2): the warp draws departures, routing and arrivals of
//     all its stations from N_{tau-1} (after the same consumer wait), publishes
//     ph1 = tau, waits for its producers' ph1 >= tau, gathers A^in, publishes
//     done = tau.
// Producers always sit at lower warp indices than their consumers, so the
// waits form no cycle.  Every wait is bounded: on timeout the warp latches an
// error bit and leaves its time loop, and warps waiting on it time out in turn.
#include <cstdint>

#include <cuda/atomic>

#include "internal.h"
#include "sampling.cuh"
#include "unit.cuh"

namespace eulernet {

namespace {

constexpr int kPipeTile = 32;             // replications per tile = lanes

__device__ __forceinline__ int load_acquire(int* p) {
  return cuda::atomic_ref<int, cuda::thread_scope_block>(*p).load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void store_release(int* p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_block>(*p).store(v, cuda::memory_order_release);
}

// Make this warp's shared-memory writes visible, then publish `tau`.
__device__ __forceinline__ void publish(int* ctr, int w, int tau, bool mute) {
  __threadfence_block();
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && !mute) store_release(ctr + w, tau);
}

// Wait until ctr[b] >= need for every warp b in `mask`, at most `limit` polls
// per warp waited on.
__device__ __forceinline__ bool wait_mask(int* ctr, unsigned mask, int need, long long limit,
                                          int sleep_ns) {
  int ok = 1;
  if (mask != 0u && need > 0 && (threadIdx.x & 31) == 0) {
    unsigned m = mask;
    while (m && ok) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      long long it = 0;
      while (load_acquire(ctr + b) < need) {
        if (++it > limit) {
          ok = 0;
          break;
        }
        if (sleep_ns > 0) __nanosleep(sleep_ns);
      }
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  __threadfence_block();
  return ok != 0;
}

// Shared layout: rinv[64] f32 | sacc[n][6] i64 | racc[32][4] i64 | ph1[32] i32 |
//                done[32] i32 | N[n][32] i32 | Redge[2][E][32] i32
template <int SCHEME>
__global__ void __launch_bounds__(512, 2) pipeline_kernel(NetTables t, RunParams p, PipePlan pp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t n = t.n, E = t.E;
  float* rinv = reinterpret_cast<float*>(smem);
  long long* sacc = reinterpret_cast<long long*>(smem + 256);
  long long* racc = sacc + 6 * (int64_t)n;
  int* ph1 = reinterpret_cast<int*>(racc + 4 * kPipeTile);
  int* done = ph1 + 32;
  int32_t* Ns = done + 32;
  int32_t* Rs = Ns + (int64_t)n * kPipeTile;
  const int64_t slot_stride = (int64_t)(E > 0 ? E : 1) * kPipeTile;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int w = tid >> 5, lane = tid & 31;
  const int k_begin = pp.wbeg[w], k_end = pp.wbeg[w + 1];
  const unsigned prod = pp.prod[w], cons = pp.cons[w];
  const bool lead = lane == 0;
  const long long lim = p.wait_limit;
  const int zz = p.wait_sleep_ns;
  const bool mute = p.test_stall != 0;

  for (int k = tid; k < 64; k += nthr) rinv[k] = k ? 1.0f / (float)k : 0.0f;
  for (int64_t k = tid; k < 6 * (int64_t)n; k += nthr) sacc[k] = 0;
  SamplerCtx cx{rinv, p.cap, 0u};
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
    const int64_t rloc = tile * kPipeTile + lane;
    const bool rvalid = rloc < p.R;
    const uint32_t rep = (uint32_t)(p.rep_begin + rloc);
    for (int64_t k = tid; k < (int64_t)n * kPipeTile; k += nthr)
      Ns[k] = t.N0 ? __ldg(t.N0 + k / kPipeTile) : 0;
    for (int k = tid; k < 4 * kPipeTile; k += nthr) racc[k] = 0;
    for (int k = tid; k < 64; k += nthr) ph1[k] = 0;  // ph1 and done
    long long q_r = 0, d_r = 0, x_r = 0, a_r = 0;
    __syncthreads();

    bool ok = true;
    for (int32_t tau = 1; tau <= p.K && ok; ++tau) {
      const float* lam_t = p.lam + (int64_t)(tau - 1) * t.n_ex;
      int32_t* slot = Rs + (tau & 1) * slot_stride;
      ok = wait_mask(done, cons, tau - 2, lim, zz);  // the buffer this step writes is free
      if (SCHEME == 1) {
        ok = ok && wait_mask(ph1, prod, tau, lim, zz);  // upstream routed counts of this step
        for (int k = k_begin; k < k_end; ++k) {
          const int32_t i = __ldg(t.lvl_station + k);
          int32_t v[5] = {0, 0, 0, 0, 0};
          if (rvalid) {
            const UnitOut o = unit_update<true>(t, p, i, (uint32_t)tau, rep, lam_t, Ns, slot,
                                                kPipeTile, lane, cx);
            const int32_t c = servers_at(t, p, i, (uint32_t)tau);
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
          reduce_to<5>(sacc + 6 * (int64_t)i, v, lead, 32, false);
        }
        publish(ph1, w, tau, mute);
        publish(done, w, tau, mute);
      } else {
        for (int k = k_begin; k < k_end; ++k) {
          const int32_t i = __ldg(t.lvl_station + k);
          int32_t v[3] = {0, 0, 0};
          if (rvalid) {
            const UnitOut o = unit_update<false>(t, p, i, (uint32_t)tau, rep, lam_t, Ns, slot,
                                                 kPipeTile, lane, cx);
            v[0] = o.D;
            v[1] = o.X;
            v[2] = o.A;
            d_r += o.D;
            x_r += o.X;
            a_r += o.A;
          }
          reduce_to<3>(sacc + 6 * (int64_t)i + 2, v, lead, 32, false);
        }
        publish(ph1, w, tau, mute);
        ok = ok && wait_mask(ph1, prod, tau, lim, zz);
        for (int k = k_begin; k < k_end; ++k) {
          const int32_t i = __ldg(t.lvl_station + k);
          int32_t v[2] = {0, 0};
          if (rvalid) {
            const int32_t nn = backward_gather(t, i, Ns, slot, kPipeTile, lane, cx.err);
            const int32_t c = servers_at(t, p, i, (uint32_t)tau);
            v[0] = nn;
            v[1] = nn < c ? nn : c;
            q_r += nn;
          }
          reduce_to<2>(sacc + 6 * (int64_t)i, v, lead, 32, false);
        }
        publish(done, w, tau, mute);
      }
    }
    if (!ok) cx.err |= kErrStall;
    __syncthreads();

    // tile epilogue: per-replication sums and N_K
    if (rvalid) {
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * lane + 0), (unsigned long long)q_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * lane + 1), (unsigned long long)d_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * lane + 2), (unsigned long long)x_r);
      atomicAdd(reinterpret_cast<unsigned long long*>(racc + 4 * lane + 3), (unsigned long long)a_r);
    }
    for (int k = k_begin; k < k_end; ++k) {
      const int32_t i = __ldg(t.lvl_station + k);
      int32_t v[1] = {rvalid ? Ns[(int64_t)i * kPipeTile + lane] : 0};
      reduce_to<1>(sacc + 6 * (int64_t)i + 5, v, lead, 32, false);
    }
    __syncthreads();
    int64_t* st_rep = p.stats + 5 * (int64_t)n;
    for (int k = tid; k < 4 * kPipeTile; k += nthr) {
      const int64_t rr = tile * kPipeTile + k / 4;
      if (rr < p.R) st_rep[rr * 4 + (k & 3)] = racc[k];
    }
    __syncthreads();
  }

  int64_t* st_nk = p.stats + 5 * (int64_t)n + 4 * p.R;
  for (int64_t k = tid; k < 6 * (int64_t)n; k += nthr) {
    const int64_t i = k / 6, s = k % 6;
    const long long v = sacc[k];
    if (v == 0) continue;
    unsigned long long* dst =
        reinterpret_cast<unsigned long long*>(s < 5 ? p.stats + i * 5 + s : st_nk + i);
    atomicAdd(dst, (unsigned long long)v);
  }
  latch(p.err, cx.err);
}

}  // namespace

int64_t pipeline_smem_bytes(int32_t n, int32_t E) {
  return 256 + 6 * 8 * (int64_t)n + 4 * 8 * kPipeTile + 2 * 32 * 4 +
         4 * ((int64_t)n + 2 * (int64_t)(E > 0 ? E : 1)) * kPipeTile;
}

cudaError_t pipeline_occupancy(int scheme, int block, int smem, int* blocks_per_sm) {
  const void* fn = scheme == 0 ? (const void*)pipeline_kernel<0> : (const void*)pipeline_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t launch_pipeline(const NetTables& t, const RunParams& p, const PipePlan& pp, int grid,
                            int smem, cudaStream_t s) {
  const void* fn = p.scheme == 0 ? (const void*)pipeline_kernel<0> : (const void*)pipeline_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int block = 32 * pp.W;
  if (p.scheme == 0)
    pipeline_kernel<0><<<grid, block, smem, s>>>(t, p, pp);
  else
    pipeline_kernel<1><<<grid, block, smem, s>>>(t, p, pp);
  return cudaGetLastError();
}

}  // namespace eulernet
