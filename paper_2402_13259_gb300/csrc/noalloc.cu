// noalloc.cu -- euler_net_simulate_noalloc: the HBM-state form of the Euler
// step run entirely out of a fixed scratch area that the library reserves
// when it is loaded, so the call itself allocates no device memory.
//
// Who needs it: programs that cannot call cudaMalloc/cudaFree while they run
// -- a host application with a device-memory budget fixed at start-up, a
// plug-in whose host owns the device allocator, or a latency-critical loop in
// which an allocation (which may synchronise the device) is not acceptable.
// They create the network handle once during set-up and then call this entry
// point; it writes into their own stats buffer.
//
// The scratch is one file-scope __device__ array (kScratchBytes, 64 MiB).
// Every GPU that loads this library holds it until the process exits.  All
// calls share it and it keeps the previous call's contents, so this file
// clears what must start at zero on every call, and calls that overlap on the
// GPU (on different streams, or from different threads) race on it.  The
// per-step tables stay in the scratch between calls: a call with the same
// handle, unchanged since, and the same (dt, T) finds them there and stages
// nothing; any other call stages them from host memory chunk by chunk and
// synchronises its stream while it does.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "handle.h"
#include "internal.h"
#include "sampling.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// The reserved scratch.  In host code this name is only a host-side stand-in
// for the device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device

// Resolve the scratch's device address once per device, with that device
// current.  The first call of the entry point on a device does this set-up.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return cudaSuccess;
}

__global__ void fold_error_kernel(const unsigned* src, unsigned* dst) {
  if (*src) atomicOr(dst, *src);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int noalloc_fail(int code, const char* msg) {
  eulernet::set_last_error(msg);
  return code;
}

// Host staging for the per-step tables: a fixed buffer, refilled chunk by
// chunk (a copy from pageable memory returns once the data is staged).
constexpr int kStage = 4096;
alignas(16) thread_local float g_stage[kStage];
thread_local int32_t g_stage_i[kStage];

// What the scratch's table area holds on each device: the tables of handle
// `uid` at generation `gen` for (dt, T).  A call that finds its own tables
// there stages nothing and does not synchronise the stream.
struct TableKey {
  uint64_t uid = 0, gen = 0;
  double dt = -1.0, T = -1.0;
};
TableKey g_tables[kMaxDevices];

}  // namespace

extern "C" EULERNET_API int euler_net_simulate_noalloc(euler_net* h, int32_t scheme, double dt,
                                                       double T, int64_t R, uint64_t seed,
                                                       int64_t rep_begin, int64_t* stats,
                                                       void* cuda_stream) {
  using namespace eulernet;
  if (!h) return noalloc_fail(EULER_ERR_ARG, "handle is NULL");
  if (scheme != EULER_BACKWARD && scheme != EULER_FORWARD) return noalloc_fail(EULER_ERR_ARG, "unknown scheme");
  if (!(dt > 0.0) || !(T > 0.0) || !std::isfinite(dt) || !std::isfinite(T))
    return noalloc_fail(EULER_ERR_ARG, "dt and T must be finite and > 0");
  if (R < 0 || rep_begin < 0 || !stats) return noalloc_fail(EULER_ERR_ARG, "bad replications, rep_begin or stats");
  if (rep_begin + R > (int64_t)1 << 32) return noalloc_fail(EULER_ERR_TOO_LARGE, "replication index beyond 2^32");
  const int64_t K = euler_num_steps(dt, T);
  if (K >= (1 << 24)) return noalloc_fail(EULER_ERR_TOO_LARGE, "too many steps (T/dt >= 2^24)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

  // scratch layout: [err, tau] | p0 constants[n] | mu h[n] | servers[K][n] (schedule only) |
  //                 lam[K][n_ex] | racc[R][4] | N[n][ld] | Redge[E][ld]
  const int64_t ld = (R + 3) / 4 * 4;
  const int64_t n_ex = h->n_ex > 0 ? h->n_ex : 1;
  size_t off = 256;
  const size_t off_p0 = off;
  off = align256(off + sizeof(float4) * (size_t)h->n);
  const size_t off_muh = off;
  off = align256(off + sizeof(float) * (size_t)h->n);
  const size_t off_mtab = off;
  if (h->sv_len > 0) off = align256(off + sizeof(int32_t) * (size_t)K * (size_t)h->n);
  const size_t off_lam = off;
  off = align256(off + sizeof(float) * (size_t)K * (size_t)n_ex);
  const size_t off_racc = off;
  off = align256(off + sizeof(int64_t) * 4 * (size_t)(R > 0 ? R : 1));
  const size_t off_N = off;
  off = align256(off + sizeof(int32_t) * (size_t)h->n * (size_t)ld);
  const size_t off_Redge = off;
  off = align256(off + sizeof(int32_t) * (size_t)(h->E > 0 ? h->E : 1) * (size_t)ld);
  if (off > kScratchBytes)
    return noalloc_fail(EULER_ERR_TOO_LARGE,
                        "this run needs more scratch than the 64 MiB the no-allocation entry point "
                        "reserves (n*R + E*R int32 state, 32 B per replication, the per-step tables)");

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return noalloc_fail(EULER_ERR_CUDA, cudaGetErrorString(e));
  if (device != h->device)
    return noalloc_fail(EULER_ERR_ARG, "the handle belongs to another device than the current one");
  unsigned char* base = nullptr;
  e = scratch_address(device, &base);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(stats, 0, sizeof(int64_t) * (size_t)euler_stats_len(h->n, R), s);
  if (e != cudaSuccess) return noalloc_fail(EULER_ERR_CUDA, cudaGetErrorString(e));
  if (R == 0) return EULER_OK;

  // per-call tables, computed by the same host functions as euler_net_simulate's
  float4* d_p0 = reinterpret_cast<float4*>(base + off_p0);
  float* d_lam = reinterpret_cast<float*>(base + off_lam);
  float* d_muh = reinterpret_cast<float*>(base + off_muh);
  int32_t* d_mtab = h->sv_len > 0 ? reinterpret_cast<int32_t*>(base + off_mtab) : nullptr;
  TableKey key;
  key.uid = h->uid;
  key.gen = h->tables_gen;
  key.dt = dt;
  key.T = T;
  TableKey& held = g_tables[device];
  const bool fresh = held.uid == key.uid && held.gen == key.gen && held.dt == key.dt && held.T == key.T;
  if (!fresh) {
    held = TableKey();  // the area is being rewritten
    for (int32_t i0 = 0; i0 < h->n && e == cudaSuccess; i0 += kStage / 5) {
      const int32_t cnt = h->n - i0 < kStage / 5 ? h->n - i0 : kStage / 5;
      step_p0(*h, dt, i0, cnt, reinterpret_cast<float4*>(g_stage), g_stage + 4 * cnt);
      e = cudaMemcpyAsync(d_p0 + i0, g_stage, sizeof(float4) * cnt, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_muh + i0, g_stage + 4 * cnt, sizeof(float) * cnt, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // staging buffer is reused
    }
    if (d_mtab) {
      // whole steps' rows per chunk (a row longer than the buffer goes alone)
      const int64_t rows = h->n <= kStage ? kStage / h->n : 0;
      for (int64_t tau = 1; tau <= K && e == cudaSuccess;) {
        if (rows > 0) {
          const int64_t cnt = K - tau + 1 < rows ? K - tau + 1 : rows;
          step_servers(*h, dt, tau, cnt, g_stage_i);
          e = cudaMemcpyAsync(d_mtab + (tau - 1) * h->n, g_stage_i, sizeof(int32_t) * (size_t)(cnt * h->n),
                              cudaMemcpyHostToDevice, s);
          tau += cnt;
        } else {
          int64_t j = (int64_t)floor((double)(tau - 1) * dt / h->sv_dt);
          if (j > h->sv_len - 1) j = h->sv_len - 1;
          e = cudaMemcpyAsync(d_mtab + (tau - 1) * h->n, h->sv_table.data() + j * h->n,
                              sizeof(int32_t) * (size_t)h->n, cudaMemcpyHostToDevice, s);
          tau += 1;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // staging buffer is reused
      }
    }
    if (h->n_ex > 0) {
      const int64_t total = K * h->n_ex;
      for (int64_t j0 = 0; j0 < total && e == cudaSuccess; j0 += kStage) {
        const int64_t cnt = total - j0 < kStage ? total - j0 : kStage;
        step_lam(*h, dt, j0, cnt, g_stage);
        e = cudaMemcpyAsync(d_lam + j0, g_stage, sizeof(float) * (size_t)cnt, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // staging buffer is reused
      }
    }
    if (e == cudaSuccess) held = key;
  }
  unsigned* d_err = reinterpret_cast<unsigned*>(base);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return noalloc_fail(EULER_ERR_CUDA, cudaGetErrorString(e));

  RunParams p;
  p.p0 = d_p0;
  p.lam = d_lam;
  p.h = (float)dt;
  p.K = (int32_t)K;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  set_round_keys(p.rk, p.key0, p.key1);
  p.R = R;
  p.rep_begin = rep_begin;
  p.scheme = scheme;
  p.tile_reps = 32;
  p.num_tiles = (R + 31) / 32;
  p.cap = h->opt[EULER_OPT_SAMPLER_CAP] > 0 ? (int32_t)h->opt[EULER_OPT_SAMPLER_CAP] : 1000;
  p.stats = stats;
  p.err = d_err;
  p.wait_limit = (int64_t)1 << 25;
  p.test_stall = 0;
  p.muh = d_muh;
  p.dep_mode = h->dep_mode();
  p.mtab = d_mtab;
  HbmState hs;
  hs.tau = reinterpret_cast<int32_t*>(base + 4);
  hs.racc = reinterpret_cast<int64_t*>(base + off_racc);
  hs.N = reinterpret_cast<int32_t*>(base + off_N);
  hs.Redge = reinterpret_cast<int32_t*>(base + off_Redge);
  hs.ld = ld;
  set_round_keys(hs, p.key0, p.key1);
  const NetTables t = h->tables();
  e = launch_hbm_init(t, p, hs, s);  // N = N0, partial sums = 0, tau = 1
  for (int64_t k = 0; k < K && e == cudaSuccess; ++k)
    e = launch_hbm_step(t, p, hs, 256, h->lvl_ptr.data(), s);
  if (e == cudaSuccess) e = launch_hbm_finish(t, p, hs, p.R, 0, s);
  if (e == cudaSuccess) {
    fold_error_kernel<<<1, 1, 0, s>>>(d_err, h->d_err);  // report through euler_net_status
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(EULER_ERR_CUDA, cudaGetErrorString(e));
  return EULER_OK;
}
