// kernels.cu -- the Euler step of arXiv 2402.13259 on sm_103a.
//
// Two forms of the same step (results identical bit for bit):
//  * persistent: one CTA owns a tile of replications, keeps the whole network
//    state of the tile (N and the routed edge counts R_e) in shared memory and
//    runs the time loop inside the kernel; CTAs loop over tiles.
//  * hbm: state in global memory (station-major, replication-fastest), one
//    kernel per phase of a step, the step loop captured in a CUDA graph; used
//    when a tile does not fit in shared memory.
//
// One "unit" is one (station, replication) update of one step:
//   backward (Sec. 2.2 tasks 1-4, Algorithm 2): D from N_{tau-1}, routing,
//     external arrivals for every station, then -- after a block barrier --
//     the gather of routed counts over the reverse graph (CSC) and the update;
//   forward (Sec. 2.2 tasks 1-4, Algorithm 3): level by level in flow order,
//     gather, external arrivals, D from N_{tau-1} + A^ex + A^in, update,
//     routing; a barrier between levels.
// Thread mapping: thread t owns replication slot r = t % Rt of the tile and
// station slots t / Rt + k G (G = blockDim / Rt), so lanes with consecutive r
// share a station: per-station sums are warp-segmented reductions and
// per-replication sums stay in registers.
#include <cstdint>

#include "internal.h"
#include "sampling.cuh"
#include "hbm_step.cuh"
#include "tile.cuh"
#include "unit.cuh"

namespace eulernet {

namespace {

// Single network: CTAs loop over the tiles.
template <int SCHEME, bool GRAD = false, bool EXT = true>
__global__ void __launch_bounds__(512, 2) persistent_kernel(NetTables t, const __grid_constant__ RunParams p) {
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
  if (GRAD) {
    const int64_t end = (int64_t)(reinterpret_cast<unsigned char*>(sm.Rs + (int64_t)t.ring * t.E * Rt) - smem);
    sm.mu_acc = reinterpret_cast<double*>(smem + (end + 15) / 16 * 16);
    sm.th_acc = sm.mu_acc + (int64_t)n * Rt;
  }
  const int tid = threadIdx.x, nthr = blockDim.x;
  fill_rinv(sm.rinv);
  for (int64_t k = tid; k < 6 * (int64_t)n; k += nthr) sm.sacc[k] = 0;
  SamplerCtx cx{sm.rinv, p.cap, 0u};
  __syncthreads();
  NoHook hook;
  for (int64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x)
    tile_body<SCHEME, GRAD, EXT>(t, p, tile, sm, cx, hook, p.rk);
  flush_station_sums(t, p, sm.sacc);
  latch(p.err, cx.err);
}

// L_m(r) S_r[c] summed over blocks of 32 consecutive replications (ascending
// inside a block): partial[b][m][c], partial sums of squares, and sums of L.
// L_1(r) = dt Q_r, L_2(r) = D_r from the per-replication statistics.
// lbar (optional, device [2]): centred estimator, terms (L - lbar[m]) S.
__global__ void grad_partial_kernel(int32_t n, int64_t R, double dt, const int64_t* stats,
                                    const double* scores, double* partial, const double* lbar) {
  const int64_t C = (int64_t)n + 3;
  const int64_t b = blockIdx.x;
  const int64_t nb = gridDim.x;
  const int64_t* rp = stats + 5 * (int64_t)n;
  double* ps = partial + b * 2 * C;             // [nb][2][C] sums
  double* pq = partial + nb * 2 * C + b * 2 * C;  // [nb][2][C] sums of squares
  double* pv = partial + 4 * nb * C + b * 2;      // [nb][2] sums of L
  for (int64_t k = threadIdx.x; k < 2 * C + 2; k += blockDim.x) {
    if (k < 2 * C) {
      const int m = (int)(k / C);
      const int64_t c = k % C;
      double s = 0.0, q = 0.0;
      for (int64_t r = b * 32; r < R && r < b * 32 + 32; ++r) {
        const double L = m == 0 ? dt * (double)rp[4 * r] : (double)rp[4 * r + 1];
        const double x = (lbar ? L - lbar[m] : L) * scores[r * C + c];
        s += x;
        q += x * x;
      }
      ps[m * C + c] = s;
      pq[m * C + c] = q;
    } else {
      const int m = (int)(k - 2 * C);
      double s = 0.0;
      for (int64_t r = b * 32; r < R && r < b * 32 + 32; ++r)
        s += m == 0 ? dt * (double)rp[4 * r] : (double)rp[4 * r + 1];
      pv[m] = s;
    }
  }
}

// Blocks summed in ascending order: grad = sum / R, value = sum L / R, and the
// variance of the mean, (sum x^2 - R g^2) / (R (R - 1)).
__global__ void grad_final_kernel(int32_t n, int64_t R, int64_t nb, const double* partial,
                                  double* grad, double* value, double* grad_var, bool write_value) {
  const int64_t C = (int64_t)n + 3;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 2 * C + 2;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < 2 * C) {
      double s = 0.0, q = 0.0;
      for (int64_t b = 0; b < nb; ++b) {
        s += partial[b * 2 * C + k];
        q += partial[nb * 2 * C + b * 2 * C + k];
      }
      const double g = s / (double)R;
      grad[k] = g;
      if (grad_var)
        grad_var[k] = R > 1 ? (q - (double)R * g * g) / ((double)R * (double)(R - 1)) : 0.0;
    } else {
      const int m = (int)(k - 2 * C);
      double s = 0.0;
      for (int64_t b = 0; b < nb; ++b) s += partial[4 * nb * C + b * 2 + m];
      if (write_value) value[m] = s / (double)R;
    }
  }
}

// Many networks: CTAs take (network, tile) work items from a queue ordered by
// decreasing cost.  Network j's tables are nets[j], its run runs[j] (tile
// size, scheme, stats buffer); per-station sums go to shared memory when the
// network's layout fits (runs[j].sacc_slot < 0) or to the CTA's slot of a
// global scratch array otherwise.
template <int SCHEME, bool EXT>
__global__ void __launch_bounds__(512, 2) batch_kernel(const NetTables* nets, const RunParams* runs,
                                                       const int2* items, int num_items,
                                                       int* next_item, long long* sacc_scratch,
                                                       int64_t sacc_slot_len) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int claim[2];
  __shared__ int s_item;
  const int tid = threadIdx.x, nthr = blockDim.x;
  float* rinv = reinterpret_cast<float*>(smem);
  fill_rinv(rinv);
  SamplerCtx cx{rinv, 1000, 0u};
  unsigned err = 0;
  unsigned* err_ptr = nullptr;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(next_item, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= num_items) break;
    const int2 wi = items[it];
    const NetTables t = nets[wi.x];
    const RunParams p = runs[wi.x];
    cx.cap = p.cap;
    err_ptr = p.err;
    const int32_t n = t.n;
    const int Rt = p.tile_reps;
    TileSmem sm;
    sm.rinv = rinv;
    unsigned char* base = smem + 256;
    if (p.sacc_in_global) {
      sm.sacc = sacc_scratch + (int64_t)blockIdx.x * sacc_slot_len;
    } else {
      sm.sacc = reinterpret_cast<long long*>(base);
      base += 8 * 6 * (int64_t)n;
    }
    sm.racc = reinterpret_cast<long long*>(base);
    sm.Ns = reinterpret_cast<int32_t*>(sm.racc + 4 * (int64_t)Rt);
    sm.Rs = sm.Ns + (int64_t)n * Rt;
    sm.claim = claim;
    for (int64_t k = tid; k < 6 * (int64_t)n; k += nthr) sm.sacc[k] = 0;
    __syncthreads();
    {
      NoHook hook;
      tile_body<SCHEME, false, EXT>(t, p, wi.y, sm, cx, hook);
    }
    flush_station_sums(t, p, sm.sacc);
    __syncthreads();
    err |= cx.err;
    cx.err = 0;
    if (err && err_ptr) {
      latch(err_ptr, err);
      err = 0;
    }
  }
}

__global__ void hbm_advance_kernel(int32_t* tau, int32_t by) { *tau += by; }

// State N_{tau0} (the network's N0, or a checkpoint), per-replication sums
// zeroed, step counter at the run's first slot tau0 + 1.
__global__ void hbm_init_kernel(NetTables t, RunParams p, HbmState hs) {
  const int64_t total = (int64_t)t.n * hs.ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / hs.ld, r = k - i * hs.ld;
    if (hs.state_in)
      hs.N[k] = r < p.R ? hs.state_in[i * hs.state_ld + hs.state_r0 + r] : 0;
    else
      hs.N[k] = t.N0 ? __ldg(t.N0 + i) : 0;
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 4 * p.R;
       k += (int64_t)gridDim.x * blockDim.x)
    hs.racc[k] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *hs.tau = p.tau0 + 1;
}

// Per-replication sums out, and N_K summed over replications (one block per
// station, 128-bit loads of the replication-fastest state).
// The replications of this call are rows r0 .. r0 + p.R of a stats layout for
// R_total replications (chunked runs); N_K accumulates over the chunks.
__global__ void hbm_finish_kernel(NetTables t, RunParams p, HbmState hs, int64_t R_total, int64_t r0) {
  int64_t* st_rep = p.stats + 5 * (int64_t)t.n + 4 * r0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 4 * p.R;
       k += (int64_t)gridDim.x * blockDim.x)
    st_rep[k] = hs.racc[k];
  __shared__ long long part[32];
  for (int32_t i = blockIdx.x; i < t.n; i += gridDim.x) {
    if (hs.state_out)  // the checkpoint N_K of this chunk's replications
      for (int64_t k = threadIdx.x; k < p.R; k += blockDim.x)
        hs.state_out[(int64_t)i * hs.state_ld + hs.state_r0 + k] = hs.N[(int64_t)i * hs.ld + k];
    const int4* row = reinterpret_cast<const int4*>(hs.N + (int64_t)i * hs.ld);
    long long s = 0;
    const int64_t nvec = p.R / 4;
    for (int64_t k = threadIdx.x; k < nvec; k += blockDim.x) {
      const int4 q = row[k];
      s += (long long)q.x + q.y + q.z + q.w;
    }
    for (int64_t k = nvec * 4 + threadIdx.x; k < p.R; k += blockDim.x) s += hs.N[(int64_t)i * hs.ld + k];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long tot = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += part[k];
      p.stats[5 * (int64_t)t.n + 4 * R_total + i] += tot;
    }
    __syncthreads();
  }
}

}  // namespace

int64_t persistent_smem_bytes(int32_t n, int32_t E, int32_t ring, int32_t tile_reps) {
  return 256 + 6 * 8 * (int64_t)n + 4 * 8 * (int64_t)tile_reps +
         4 * ((int64_t)n + (int64_t)ring * E) * tile_reps;
}

namespace {
bool uses_ext(const RunParams& p) { return p.mtab != nullptr || p.dep_mode != 0; }

template <bool GRAD>
const void* persistent_fn(int scheme, bool ext) {
  if (scheme == 0)
    return ext ? (const void*)persistent_kernel<0, GRAD, true> : (const void*)persistent_kernel<0, GRAD, false>;
  return ext ? (const void*)persistent_kernel<1, GRAD, true> : (const void*)persistent_kernel<1, GRAD, false>;
}

const void* batch_fn(int scheme, bool ext) {
  if (scheme == 0) return ext ? (const void*)batch_kernel<0, true> : (const void*)batch_kernel<0, false>;
  return ext ? (const void*)batch_kernel<1, true> : (const void*)batch_kernel<1, false>;
}

// Occupancy of the tightest of a set of instantiations at (block, smem).
cudaError_t min_occupancy(const void* const* fns, int count, int block, int smem, int* blocks_per_sm) {
  int best = 1 << 30;
  for (int k = 0; k < count; ++k) {
    cudaError_t e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int v = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fns[k], block, smem);
    if (e != cudaSuccess) return e;
    best = v < best ? v : best;
  }
  *blocks_per_sm = best;
  return cudaSuccess;
}

cudaError_t launch_fn(const void* fn, void** args, int grid, int block, int smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, (size_t)smem, s);
}
}  // namespace

cudaError_t persistent_occupancy(int scheme, int block, int smem, int* blocks_per_sm) {
  const void* fns[2] = {persistent_fn<false>(scheme, false), persistent_fn<false>(scheme, true)};
  return min_occupancy(fns, 2, block, smem, blocks_per_sm);
}

cudaError_t launch_persistent(const NetTables& t, const RunParams& p, int grid, int block, int smem,
                              cudaStream_t s) {
  NetTables tt = t;
  RunParams pp = p;
  void* args[] = {&tt, &pp};
  return launch_fn(persistent_fn<false>(p.scheme, uses_ext(p)), args, grid, block, smem, s);
}

cudaError_t batch_occupancy(int block, int smem, int* blocks_per_sm) {
  const void* fns[4] = {batch_fn(0, false), batch_fn(1, false), batch_fn(0, true), batch_fn(1, true)};
  return min_occupancy(fns, 4, block, smem, blocks_per_sm);
}

cudaError_t launch_batch(int scheme, bool ext, const NetTables* nets, const RunParams* runs,
                         const int2* items, int num_items, int* next_item, long long* sacc_scratch,
                         int64_t sacc_slot_len, int grid, int block, int smem, cudaStream_t s) {
  void* args[] = {&nets, &runs, &items, &num_items, &next_item, &sacc_scratch, &sacc_slot_len};
  return launch_fn(batch_fn(scheme, ext), args, grid, block, smem, s);
}

int64_t grad_smem_extra(int32_t n, int32_t n_ex, int32_t tile_reps) {
  return 16 + 8 * ((int64_t)n + 3 * (int64_t)n_ex) * tile_reps;
}

cudaError_t grad_occupancy(int scheme, int block, int smem, int* blocks_per_sm) {
  const void* fns[2] = {persistent_fn<true>(scheme, false), persistent_fn<true>(scheme, true)};
  return min_occupancy(fns, 2, block, smem, blocks_per_sm);
}

cudaError_t launch_persistent_grad(const NetTables& t, const RunParams& p, int grid, int block,
                                   int smem, cudaStream_t s) {
  NetTables tt = t;
  RunParams pp = p;
  void* args[] = {&tt, &pp};
  return launch_fn(persistent_fn<true>(p.scheme, uses_ext(p)), args, grid, block, smem, s);
}

cudaError_t launch_grad_reduce(int32_t n, int64_t R, double dt, const int64_t* stats,
                               const double* scores, double* partial, double* grad, double* value,
                               double* grad_var, bool center, cudaStream_t s) {
  const int64_t nb = (R + 31) / 32;
  grad_partial_kernel<<<(unsigned)nb, 128, 0, s>>>(n, R, dt, stats, scores, partial, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grad_final_kernel<<<8, 128, 0, s>>>(n, R, nb, partial, grad, value, grad_var, true);
  e = cudaGetLastError();
  if (e != cudaSuccess || !center) return e;
  // centred estimator: a second pass with the value just computed
  grad_partial_kernel<<<(unsigned)nb, 128, 0, s>>>(n, R, dt, stats, scores, partial, value);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grad_final_kernel<<<8, 128, 0, s>>>(n, R, nb, partial, grad, value, grad_var, false);
  return cudaGetLastError();
}

namespace {
__global__ void average_kernel(const int64_t* b, const int64_t* f, double* out, int64_t len) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = 0.5 * ((double)b[k] + (double)f[k]);
}
}  // namespace

cudaError_t launch_average(const int64_t* b, const int64_t* f, double* out, int64_t len,
                           cudaStream_t s) {
  average_kernel<<<256, 256, 0, s>>>(b, f, out, len);
  return cudaGetLastError();
}

int64_t hbm_smem_bytes(int32_t, int32_t) { return 0; }

cudaError_t launch_hbm_init(const NetTables& t, const RunParams& p, const HbmState& hs,
                            cudaStream_t s) {
  hbm_init_kernel<<<1024, 256, 0, s>>>(t, p, hs);
  return cudaGetLastError();
}

cudaError_t launch_hbm_step(const NetTables& t, const RunParams& p, const HbmState& hs, int block,
                            const int32_t* lvl_ptr_host, cudaStream_t s) {
  const int G = block / kHbmTile;
  const unsigned tiles = (unsigned)((p.R + kHbmTile - 1) / kHbmTile);
  if (p.scheme == 0) {
    dim3 grid(tiles, (unsigned)((t.n + G - 1) / G));
    hbm_phase_kernel<0><<<grid, block, 0, s>>>(t, p, hs, 0, t.n, 0);
    hbm_phase_kernel<1><<<grid, block, 0, s>>>(t, p, hs, 0, t.n, 0);
  } else {
    for (int32_t j = 0; j < t.L; ++j) {
      const int32_t s0 = lvl_ptr_host[j], m = lvl_ptr_host[j + 1] - lvl_ptr_host[j];
      dim3 grid(tiles, (unsigned)((m + G - 1) / G));
      hbm_phase_kernel<2><<<grid, block, 0, s>>>(t, p, hs, s0, m, 0);
    }
  }
  hbm_advance_kernel<<<1, 1, 0, s>>>(hs.tau, 1);
  return cudaGetLastError();
}

namespace {
// Slot kernels are launched with programmatic stream serialisation: a slot's
// CTAs may start (and fill their 1/k tables) while the previous slot's last
// CTAs finish; each waits for the previous grid's completion and memory
// (griddepcontrol.wait) before it reads the state.
template <bool GRAD, bool SOJ>
cudaError_t launch_slot_kernel(const NetTables& t, const RunParams& p, const HbmState& hs, dim3 grid,
                               int block, int32_t koff, bool ext, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int32_t s0 = 0, m = t.n;
  if (p.scheme == 0)
    return ext ? cudaLaunchKernelEx(&cfg, hbm_phase_kernel<4, true, GRAD, SOJ>, t, p, hs, s0, m, koff)
               : cudaLaunchKernelEx(&cfg, hbm_phase_kernel<4, false, GRAD, SOJ>, t, p, hs, s0, m, koff);
  return ext ? cudaLaunchKernelEx(&cfg, hbm_phase_kernel<3, true, GRAD, SOJ>, t, p, hs, s0, m, koff)
             : cudaLaunchKernelEx(&cfg, hbm_phase_kernel<3, false, GRAD, SOJ>, t, p, hs, s0, m, koff);
}

__global__ void hbm_sojourn_init_kernel(RunParams p, HbmState hs, int32_t station, int32_t tau0) {
  const int64_t total = (int64_t)hs.S * hs.ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    hs.cloc[k] = soj_pack(station, tau0, true);
    hs.cpos[k] = 0;
    hs.csteps[k] = 0;
  }
}

__global__ void hbm_sojourn_finish_kernel(RunParams p, HbmState hs, int32_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.R * hs.S;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / hs.S, c = k % hs.S;
    const int64_t ci = c * hs.ld + r;
    const int32_t st = hs.csteps[ci];
    out[k] = hs.cloc[ci] == kSojDone ? st : -st;
  }
}

// S_r: mu_i sums, then (a, b, phase) summed over external stations in order.
__global__ void hbm_scores_kernel(NetTables t, RunParams p, HbmState hs) {
  const int64_t C = (int64_t)t.n + 3;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.R * C;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / C, c = k % C;
    double v;
    if (c < t.n) {
      v = hs.mu_acc[c * hs.ld + r];
    } else {
      v = 0.0;
      for (int32_t ec = 0; ec < t.n_ex; ++ec) v += hs.th_acc[((int64_t)ec * 3 + (c - t.n)) * hs.ld + r];
    }
    p.scores[k] = v;
  }
}
}  // namespace

cudaError_t launch_hbm_slot(const NetTables& t, const RunParams& p, const HbmState& hs, int block,
                            int32_t koff, int mode, cudaStream_t s) {
  const int G = block / kHbmTile;  // stations per block
  const unsigned tiles = (unsigned)((p.R + kHbmTile - 1) / kHbmTile);
  dim3 grid(tiles, (unsigned)((t.n + G - 1) / G));
  const bool ext = p.mtab != nullptr || p.dep_mode != 0;
  if (mode == kHbmGrad) return launch_slot_kernel<true, false>(t, p, hs, grid, block, koff, ext, s);
  if (mode == kHbmSojourn) return launch_slot_kernel<false, true>(t, p, hs, grid, block, koff, ext, s);
  return launch_slot_kernel<false, false>(t, p, hs, grid, block, koff, ext, s);
}

cudaError_t launch_hbm_sojourn_init(const RunParams& p, const HbmState& hs, int32_t station,
                                    int32_t tau0, cudaStream_t s) {
  hbm_sojourn_init_kernel<<<512, 256, 0, s>>>(p, hs, station, tau0);
  return cudaGetLastError();
}

cudaError_t launch_hbm_sojourn_finish(const RunParams& p, const HbmState& hs, int32_t* out,
                                      cudaStream_t s) {
  hbm_sojourn_finish_kernel<<<512, 256, 0, s>>>(p, hs, out);
  return cudaGetLastError();
}

cudaError_t launch_hbm_scores(const NetTables& t, const RunParams& p, const HbmState& hs,
                              cudaStream_t s) {
  hbm_scores_kernel<<<1024, 256, 0, s>>>(t, p, hs);
  return cudaGetLastError();
}

cudaError_t launch_hbm_advance(const HbmState& hs, int32_t by, cudaStream_t s) {
  hbm_advance_kernel<<<1, 1, 0, s>>>(hs.tau, by);
  return cudaGetLastError();
}

cudaError_t launch_hbm_finish(const NetTables& t, const RunParams& p, const HbmState& hs,
                              int64_t R_total, int64_t r0, cudaStream_t s) {
  hbm_finish_kernel<<<t.n < 1024 ? t.n : 1024, 256, 0, s>>>(t, p, hs, R_total, r0);
  return cudaGetLastError();
}

}  // namespace eulernet
