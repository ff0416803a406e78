// batch.cu -- many independent networks (uneven sizes and horizons) in one
// persistent launch fed by a work queue, planned and autotuned on the host and
// replayed from a CUDA graph.
//
// Two kinds of networks.  A network with n_j R_j >= hbm_min_units units per
// step fills the GPU by itself: it runs in the HBM form, the per-step kernels
// of euler_net_simulate (one warp per station and 32 replications, a CUDA
// graph of slots replayed to its horizon), one such network after another.
// The others share one persistent launch fed by a work queue.
//
// Work item = (network j, tile of replications).  Network j gets a tile size
// Rt_j (a power of two) so that its widest phase keeps the block busy
// (forward: widest level x Rt_j ~ block; backward: all stations), scaled by
// 2^rt_shift, reduced until its tile's state fits the shared-memory budget;
// its per-station accumulators go to a global scratch slot of the CTA when
// they do not fit.  Items are sorted by decreasing cost n_j K_j Rt_j so the
// last CTAs to finish take the cheapest items.
//
// The autotuner searches the persistent launch's threads per block (stations
// per CTA), shared-memory budget and tile scale (replications per tile), the
// HBM form's threads per block and slots per graph replay (steps per
// launch), and the n R threshold between the two kinds.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "handle.h"
#include "internal.h"

using namespace eulernet;

struct euler_batch {
  int32_t count = 0;
  std::vector<euler_net*> nets;
  std::vector<euler_run> runs;
  int device = 0, sm_count = 0, smem_optin = 0;
  // networks run in the HBM form, and its launch shape
  std::vector<int> hbm_nets;
  std::vector<char> is_hbm;  // per network
  int64_t hbm_min_units = kHbmMinUnitsPerStep;
  double cp_factor = 1.0;  // critical-path rule (see make_batch_plan); <= 0 off
  int hbm_block = kHbmBlock;
  int hbm_graph_steps = 32;
  int rt_shift = 0;  // persistent tiles scaled by 2^rt_shift
  // current plan
  int block = 256;
  int64_t smem_cap = 0;  // shared-memory budget per CTA used by the plan
  int grid = 0;
  int smem = 0;
  int num_items = 0;
  int num_items_s[2] = {0, 0};  // items of each scheme: [0, n0) backward, [n0, n) forward
  int64_t sacc_slot_len = 0;
  std::vector<RunParams> h_runs;
  std::vector<NetTables> h_nets;
  std::vector<int2> h_items;
  NetTables* d_nets = nullptr;
  RunParams* d_runs = nullptr;
  int2* d_items = nullptr;
  size_t items_cap = 0;
  int* d_counter = nullptr;
  long long* d_sacc = nullptr;
  size_t sacc_cap = 0;
  // graph of the last run
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t*> graph_stats;
  cudaStream_t cap_stream = nullptr;
};

namespace {

int bfail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

int bcuda(cudaError_t e, const char* where) {
  std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  set_last_error(m.c_str());
  return e == cudaErrorMemoryAllocation ? EULER_ERR_OOM : EULER_ERR_CUDA;
}

#define BTRY(expr)                                  \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return bcuda(e_, #expr); \
  } while (0)

int64_t pow2_floor(int64_t v) {
  int64_t p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

int64_t state_bytes(const euler_net* h, int64_t Rt) {
  return 32 * Rt + 4 * ((int64_t)h->n + (int64_t)h->tables().ring * h->E) * Rt;
}

bool runs_hbm(const euler_batch* b, int j) { return b->is_hbm[j] != 0; }

// Tile of network j in the persistent launch: the widest phase x Rt ~ block,
// scaled by 2^rt_shift, reduced until it fits the budget (per-station sums in
// shared memory if possible, else in the CTA's global slot).
bool tile_for(const euler_batch* b, int j, int block, int64_t cap, int rt_shift, int64_t* Rt_out,
              bool* sacc_global_out) {
  const euler_net* h = b->nets[j];
  const int64_t width = b->runs[j].scheme == EULER_BACKWARD ? h->n : h->max_level;
  int64_t Rt = std::max<int64_t>(32, pow2_floor(std::max<int64_t>(block / std::max<int64_t>(width, 1), 1)));
  Rt = rt_shift >= 0 ? Rt << rt_shift : Rt >> -rt_shift;
  Rt = std::max<int64_t>(1, std::min<int64_t>(Rt, block));
  const int64_t sacc_bytes = 48 * (int64_t)h->n;
  for (; Rt >= 1; Rt /= 2) {
    if (256 + sacc_bytes + state_bytes(h, Rt) <= cap) {
      *Rt_out = Rt;
      *sacc_global_out = false;
      return true;
    }
    if (256 + state_bytes(h, Rt) <= cap) {
      *Rt_out = Rt;
      *sacc_global_out = true;
      return true;
    }
  }
  return false;
}

// Plan for a block size, a per-CTA shared-memory budget, a tile scale, the
// HBM-form threshold and the critical-path factor.
//
// Critical-path rule: a work item is one tile of replications through the
// network's whole horizon on one CTA, so when the launch has more items than
// CTAs, a network whose item costs (n K Rt) more than cp_factor x the mean
// load per CTA (sum of n K R over the launch's networks / CTAs) would outlast
// the rest of the launch; such a network runs in the HBM form instead, where
// one step of all its replications spreads over the whole GPU, provided a
// step has at least 2^14 units (512 warps) so that its launches do more than
// wait on launch latency.  With fewer items than CTAs every item runs at
// once and nothing moves.
int make_batch_plan(euler_batch* b, int block, int64_t cap, int rt_shift, int64_t hbm_min_units,
                    double cp_factor) {
  if (block % 32 || block < 32 || block > 512) return bfail(EULER_ERR_ARG, "batch block must be a multiple of 32 in [32, 512]");
  cap = std::min<int64_t>(cap, b->smem_optin);
  b->block = block;
  b->smem_cap = cap;
  b->rt_shift = rt_shift;
  b->hbm_min_units = hbm_min_units;
  b->cp_factor = cp_factor;
  b->is_hbm.assign(b->count, 0);
  for (int j = 0; j < b->count; ++j)
    b->is_hbm[j] = hbm_min_units > 0 && (int64_t)b->nets[j]->n * b->runs[j].replications >= hbm_min_units;
  std::vector<int64_t> Rt_of(b->count, 1);
  std::vector<char> sacc_g(b->count, 0);
  for (int j = 0; j < b->count; ++j) {
    if (b->is_hbm[j]) continue;
    bool g = false;
    if (!tile_for(b, j, block, cap, rt_shift, &Rt_of[j], &g))
      return bfail(EULER_ERR_TOO_LARGE, "a network's smallest tile does not fit the shared-memory budget");
    sacc_g[j] = g;
  }
  if (cp_factor > 0.0) {
    for (int pass = 0; pass < 8; ++pass) {
      int64_t smem = 256;
      double work = 0.0, n_items = 0.0;
      for (int j = 0; j < b->count; ++j) {
        if (b->is_hbm[j]) continue;
        const euler_net* h = b->nets[j];
        smem = std::max<int64_t>(smem, 256 + (sacc_g[j] ? 0 : 48 * (int64_t)h->n) + state_bytes(h, Rt_of[j]));
        work += (double)h->n * (double)euler_num_steps(b->runs[j].dt, b->runs[j].T) * (double)b->runs[j].replications;
        n_items += (double)((b->runs[j].replications + Rt_of[j] - 1) / Rt_of[j]);
      }
      int per_sm = 0;
      BTRY(batch_occupancy(block, (int)smem, &per_sm));
      const double ctas = std::max(1.0, (double)per_sm * b->sm_count);
      if (n_items <= ctas) break;
      bool moved = false;
      for (int j = 0; j < b->count; ++j) {
        if (b->is_hbm[j] || (int64_t)b->nets[j]->n * b->runs[j].replications < (int64_t(1) << 14)) continue;
        const double item = (double)b->nets[j]->n * (double)euler_num_steps(b->runs[j].dt, b->runs[j].T) * (double)Rt_of[j];
        if (item > cp_factor * work / ctas) {
          b->is_hbm[j] = 1;
          moved = true;
        }
      }
      if (!moved) break;
    }
  }
  b->hbm_nets.clear();
  b->h_runs.assign(b->count, RunParams{});
  b->h_nets.assign(b->count, NetTables{});
  b->h_items.clear();
  int64_t smem = 256, slot = 0;
  struct Cost { double c; int j; int64_t tile; };
  std::vector<Cost> items;
  for (int j = 0; j < b->count; ++j) {
    euler_net* h = b->nets[j];
    const euler_run& r = b->runs[j];
    const int64_t K = euler_num_steps(r.dt, r.T);
    if (b->is_hbm[j]) {
      b->hbm_nets.push_back(j);
      continue;
    }
    const int64_t Rt = Rt_of[j];
    const bool sacc_global = sacc_g[j] != 0;
    const int64_t sacc_bytes = 48 * (int64_t)h->n;
    smem = std::max<int64_t>(smem, 256 + (sacc_global ? 0 : sacc_bytes) + state_bytes(h, Rt));
    if (sacc_global) slot = std::max<int64_t>(slot, 6 * (int64_t)h->n);
    RunParams p;
    std::memset(&p, 0, sizeof p);
    p.p0 = h->d_p0;
    p.lam = h->d_lam;
    p.h = (float)r.dt;
    p.K = (int32_t)K;
    p.key0 = (uint32_t)r.seed;
    p.key1 = (uint32_t)(r.seed >> 32);
    set_round_keys(p.rk, p.key0, p.key1);
    p.R = r.replications;
    p.rep_begin = r.rep_begin;
    p.scheme = r.scheme;
    p.tile_reps = (int32_t)Rt;
    p.num_tiles = (r.replications + Rt - 1) / Rt;
    p.cap = h->opt[EULER_OPT_SAMPLER_CAP] > 0 ? (int32_t)h->opt[EULER_OPT_SAMPLER_CAP] : 1000;
    p.stats = nullptr;
    p.err = h->d_err;
    p.wait_limit = (int64_t)1 << 25;
    p.test_stall = 0;
    p.sacc_in_global = sacc_global ? 1 : 0;
    p.muh = h->d_muh;
    p.dep_mode = h->dep_mode();
    p.mtab = h->mtab();
    b->h_runs[j] = p;
    b->h_nets[j] = h->tables();
    const double c = (double)h->n * (double)K * (double)Rt;
    for (int64_t tile = 0; tile < p.num_tiles; ++tile) items.push_back({c, j, tile});
  }
  // backward items first, then forward; each group by decreasing cost
  std::stable_sort(items.begin(), items.end(), [&](const Cost& a, const Cost& c) {
    const int sa = b->runs[a.j].scheme, sc = b->runs[c.j].scheme;
    return sa != sc ? sa < sc : a.c > c.c;
  });
  b->num_items_s[0] = b->num_items_s[1] = 0;
  for (const Cost& it : items) b->num_items_s[b->runs[it.j].scheme]++;
  if (items.size() > (size_t)INT32_MAX) return bfail(EULER_ERR_TOO_LARGE, "too many work items");
  for (const Cost& it : items) b->h_items.push_back(make_int2(it.j, (int)it.tile));
  b->num_items = (int)items.size();
  b->smem = (int)smem;
  b->sacc_slot_len = slot;
  int per_sm = 0;
  BTRY(batch_occupancy(block, b->smem, &per_sm));
  if (per_sm < 1 && b->num_items > 0) return bfail(EULER_ERR_TOO_LARGE, "batch kernel cannot be resident");
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * b->sm_count, std::max(b->num_items, 1)));
  // device copies
  if (!b->d_nets) BTRY(cudaMalloc(&b->d_nets, sizeof(NetTables) * std::max(b->count, 1)));
  if (!b->d_runs) BTRY(cudaMalloc(&b->d_runs, sizeof(RunParams) * std::max(b->count, 1)));
  if (!b->d_counter) BTRY(cudaMalloc(&b->d_counter, 2 * sizeof(int)));
  if ((size_t)b->num_items > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    BTRY(cudaMalloc(&b->d_items, sizeof(int2) * std::max(b->num_items, 1)));
    b->items_cap = b->num_items;
  }
  const size_t sacc_need = (size_t)b->grid * (size_t)slot;
  if (sacc_need > b->sacc_cap) {
    cudaFree(b->d_sacc);
    b->d_sacc = nullptr;
    BTRY(cudaMalloc(&b->d_sacc, sizeof(long long) * sacc_need));
    b->sacc_cap = sacc_need;
  }
  BTRY(cudaMemcpy(b->d_nets, b->h_nets.data(), sizeof(NetTables) * b->count, cudaMemcpyHostToDevice));
  if (b->num_items)
    BTRY(cudaMemcpy(b->d_items, b->h_items.data(), sizeof(int2) * b->num_items, cudaMemcpyHostToDevice));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->graph_stats.clear();
  return EULER_OK;
}

// Steps of network j in a tuning run whose horizons are all scaled by
// k_scale (every network keeps at least one step), or its K if k_scale <= 0.
int64_t scaled_steps(const euler_batch* b, int j, double k_scale) {
  const int64_t K = euler_num_steps(b->runs[j].dt, b->runs[j].T);
  if (k_scale <= 0.0) return K;
  return std::max<int64_t>(1, std::min<int64_t>(K, (int64_t)ceil((double)K * k_scale)));
}

// Upload the run table with these stats pointers (horizons scaled by k_scale
// for tuning, see scaled_steps).
int upload_runs(euler_batch* b, int64_t* const* stats, double k_scale) {
  std::vector<RunParams> rp = b->h_runs;
  for (int j = 0; j < b->count; ++j) {
    rp[j].stats = stats[j];
    if (!b->is_hbm[j]) rp[j].K = (int32_t)scaled_steps(b, j, k_scale);
  }
  BTRY(cudaMemcpy(b->d_runs, rp.data(), sizeof(RunParams) * b->count, cudaMemcpyHostToDevice));
  return EULER_OK;
}

// The networks of the HBM form, one after another on stream s (horizons
// scaled by k_scale for tuning; only the networks in `subset` when it is not
// null).
int run_hbm_nets(euler_batch* b, int64_t* const* stats, cudaStream_t s, double k_scale,
                 const std::vector<int>* subset = nullptr) {
  for (int j : subset ? *subset : b->hbm_nets) {
    const euler_run& r = b->runs[j];
    const int rc = simulate_hbm(b->nets[j], r.scheme, r.dt, r.T, r.replications, r.seed, r.rep_begin, stats[j], s,
                                b->hbm_block, b->hbm_graph_steps, k_scale > 0.0 ? scaled_steps(b, j, k_scale) : 0);
    if (rc) return rc;
  }
  return EULER_OK;
}

// Zero the queue counter and every stats buffer, then launch (capturable).
cudaError_t enqueue(euler_batch* b, int64_t* const* stats, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int), s);
  for (int j = 0; j < b->count && e == cudaSuccess; ++j)
    e = cudaMemsetAsync(stats[j], 0,
                        sizeof(int64_t) * (size_t)euler_stats_len(b->nets[j]->n, b->runs[j].replications), s);
  bool ext = false;
  for (const RunParams& rp : b->h_runs) ext = ext || rp.mtab != nullptr || rp.dep_mode != 0;
  int off = 0;
  for (int sc = 0; sc < 2 && e == cudaSuccess; ++sc) {
    if (b->num_items_s[sc] > 0)
      e = launch_batch(sc, ext, b->d_nets, b->d_runs, b->d_items + off, b->num_items_s[sc], b->d_counter + sc,
                       b->d_sacc, b->sacc_slot_len, b->grid, b->block, b->smem, s);
    off += b->num_items_s[sc];
  }
  return e;
}

}  // namespace

extern "C" {

int euler_batch_create(euler_batch** out, euler_net* const* nets, const euler_run* runs,
                       int32_t count) try {
  if (!out) return bfail(EULER_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 0 || (count > 0 && (!nets || !runs))) return bfail(EULER_ERR_ARG, "bad batch arguments");
  euler_batch* b = new euler_batch();
  b->count = count;
  b->nets.assign(nets, nets + count);
  b->runs.assign(runs, runs + count);
  for (int j = 0; j < count; ++j) {
    const euler_run& r = runs[j];
    if (!nets[j] || (r.scheme != EULER_BACKWARD && r.scheme != EULER_FORWARD) || !(r.dt > 0.0) ||
        !(r.T > 0.0) || !std::isfinite(r.dt) || !std::isfinite(r.T) || r.replications < 0 ||
        r.rep_begin < 0 || r.rep_begin + r.replications > ((int64_t)1 << 32) ||
        euler_num_steps(r.dt, r.T) >= (1 << 24)) {
      delete b;
      return bfail(EULER_ERR_ARG, "bad run " + std::to_string(j));
    }
    for (int k = 0; k < j; ++k)
      if (nets[k] == nets[j] && (runs[k].dt != r.dt || runs[k].T != r.T)) {
        delete b;
        return bfail(EULER_ERR_ARG, "a handle appears twice with different (dt, T)");
      }
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  if (e != cudaSuccess) {
    delete b;
    return bcuda(e, "euler_batch_create device query");
  }
  for (int j = 0; j < count; ++j) {
    int rc = prepare_step_tables(nets[j], runs[j].dt, runs[j].T, nullptr);
    if (rc) {
      euler_batch_destroy(b);
      return rc;
    }
  }
  int rc = make_batch_plan(b, 256, 110 * 1024, 0, kHbmMinUnitsPerStep, 1.0);
  if (rc) {
    euler_batch_destroy(b);
    return rc;
  }
  *out = b;
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return bfail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return bfail(EULER_ERR_CUDA, "unexpected error");
}

int euler_batch_autotune(euler_batch* b, void* cuda_stream, int32_t* block_out) try {
  if (!b) return bfail(EULER_ERR_ARG, "batch is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // scratch stats buffers for the trial runs
  std::vector<int64_t*> st(b->count, nullptr);
  size_t total = 0;
  for (int j = 0; j < b->count; ++j) total += (size_t)euler_stats_len(b->nets[j]->n, b->runs[j].replications);
  int64_t* pool = nullptr;
  BTRY(cudaMalloc(&pool, sizeof(int64_t) * std::max<size_t>(total, 1)));
  size_t off = 0;
  for (int j = 0; j < b->count; ++j) {
    st[j] = pool + off;
    off += (size_t)euler_stats_len(b->nets[j]->n, b->runs[j].replications);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = EULER_OK;
  // Trials run every horizon scaled by one factor (the longest to 48 steps),
  // so that work items keep their relative lengths (the critical path).
  int64_t kmax = 1;
  for (int j = 0; j < b->count; ++j) kmax = std::max<int64_t>(kmax, euler_num_steps(b->runs[j].dt, b->runs[j].T));
  const double k_scale = std::min(1.0, 48.0 / (double)kmax);
  // one timed trial: the persistent launch and, if hbm, the HBM-form
  // networks (`subset` only, if set), horizons scaled by ks
  auto trial = [&](double ks, bool persistent, bool hbm, const std::vector<int>* subset, float* ms) -> int {
    int r = upload_runs(b, st.data(), ks);
    if (r) return r;
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess && persistent && b->num_items > 0) e = enqueue(b, st.data(), s);
    if (e != cudaSuccess) return bcuda(e, "batch autotune");
    if (hbm) {
      r = run_hbm_nets(b, st.data(), s, ks, subset);
      if (r) return r;
    }
    e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e == cudaSuccess ? EULER_OK : bcuda(e, "batch autotune");
  };
  const int64_t hbm_min0 = b->hbm_min_units;
  const double cp0 = b->cp_factor;
  int best_block = b->block, best_shift = b->rt_shift;
  int64_t best_cap = b->smem_cap, best_min = hbm_min0;
  double best_cp = cp0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = bcuda(cudaErrorUnknown, "event");
  // 1. the persistent launch: threads per block x shared-memory budget x tile scale
  {
    const int blocks[3] = {128, 256, 512};
    const int64_t caps[3] = {72 * 1024, 110 * 1024, 227 * 1024};
    float best = -1.0f;
    for (int bi = 0; bi < 3 && rc == EULER_OK; ++bi)
      for (int ci = 0; ci < 3 && rc == EULER_OK; ++ci)
        for (int sh = -1; sh <= 1 && rc == EULER_OK; ++sh) {
          if (make_batch_plan(b, blocks[bi], caps[ci], sh, hbm_min0, cp0) != EULER_OK || b->num_items == 0) continue;
          float ms = 0.0f;
          rc = trial(k_scale, true, false, nullptr, &ms);
          if (rc == EULER_OK && (best < 0.0f || ms < best)) {
            best = ms;
            best_block = blocks[bi];
            best_cap = caps[ci];
            best_shift = sh;
          }
        }
  }
  // 2. the HBM form: threads per step kernel x slots per graph replay, on up
  // to six of its networks spread over their sizes, 128 steps each at most
  if (rc == EULER_OK) rc = make_batch_plan(b, best_block, best_cap, best_shift, hbm_min0, cp0);
  if (rc == EULER_OK && !b->hbm_nets.empty()) {
    std::vector<int> by_size = b->hbm_nets;
    std::sort(by_size.begin(), by_size.end(), [&](int x, int y) {
      return b->nets[x]->n * b->runs[x].replications < b->nets[y]->n * b->runs[y].replications;
    });
    std::vector<int> sample;
    const size_t m = std::min<size_t>(6, by_size.size());
    for (size_t k = 0; k < m; ++k) sample.push_back(by_size[(k * (by_size.size() - 1)) / std::max<size_t>(m - 1, 1)]);
    int64_t ks_max = 1;
    for (int j : sample) ks_max = std::max<int64_t>(ks_max, euler_num_steps(b->runs[j].dt, b->runs[j].T));
    const double ks2 = std::min(1.0, 128.0 / (double)ks_max);
    const int hblocks[2] = {128, 256};
    const int gsteps[3] = {16, 32, 64};
    float best = -1.0f;
    int bb = b->hbm_block, bg = b->hbm_graph_steps;
    for (int bi = 0; bi < 2 && rc == EULER_OK; ++bi)
      for (int gi = 0; gi < 3 && rc == EULER_OK; ++gi) {
        b->hbm_block = hblocks[bi];
        b->hbm_graph_steps = gsteps[gi];
        float ms = 0.0f;
        rc = trial(ks2, false, true, &sample, &ms);
        if (rc == EULER_OK && (best < 0.0f || ms < best)) {
          best = ms;
          bb = hblocks[bi];
          bg = gsteps[gi];
        }
      }
    b->hbm_block = bb;
    b->hbm_graph_steps = bg;
  }
  // 3. which networks take the HBM form: the n R threshold x the
  // critical-path rule (on / off), the whole batch
  if (rc == EULER_OK) {
    const int64_t mins[4] = {int64_t(1) << 16, int64_t(1) << 18, int64_t(1) << 20, 0};
    const double cps[2] = {1.0, 0.0};
    float best = -1.0f;
    for (int mi = 0; mi < 4 && rc == EULER_OK; ++mi)
      for (int ci = 0; ci < 2 && rc == EULER_OK; ++ci) {
        if (make_batch_plan(b, best_block, best_cap, best_shift, mins[mi], cps[ci]) != EULER_OK) continue;
        float ms = 0.0f;
        rc = trial(k_scale, true, true, nullptr, &ms);
        if (rc == EULER_OK && (best < 0.0f || ms < best)) {
          best = ms;
          best_min = mins[mi];
          best_cp = cps[ci];
        }
      }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(pool);
  for (euler_net* h : b->nets) cudaMemset(h->d_err, 0, sizeof(unsigned));
  if (rc) return rc;
  rc = make_batch_plan(b, best_block, best_cap, best_shift, best_min, best_cp);
  if (rc) return rc;
  if (block_out) *block_out = b->block;
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return bfail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return bfail(EULER_ERR_CUDA, "unexpected error");
}

int euler_batch_run(euler_batch* b, int64_t* const* stats, void* cuda_stream) try {
  if (!b || (b->count > 0 && !stats)) return bfail(EULER_ERR_ARG, "bad batch run arguments");
  for (int j = 0; j < b->count; ++j)
    if (!stats[j]) return bfail(EULER_ERR_ARG, "a stats pointer is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // the handles' per-step tables for the batch's (dt, T): another call on a
  // handle since the plan may have rebuilt them elsewhere
  bool moved = false;
  for (int j = 0; j < b->count; ++j) {
    euler_net* h = b->nets[j];
    const int rc = prepare_step_tables(h, b->runs[j].dt, b->runs[j].T, s);
    if (rc) return rc;
    RunParams& p = b->h_runs[j];
    if (!runs_hbm(b, j) && (p.p0 != h->d_p0 || p.lam != h->d_lam || p.muh != h->d_muh || p.mtab != h->mtab())) {
      p.p0 = h->d_p0;
      p.lam = h->d_lam;
      p.muh = h->d_muh;
      p.mtab = h->mtab();
      moved = true;
    }
  }
  const bool same = !moved && b->exec && b->graph_stats.size() == (size_t)b->count &&
                    std::equal(b->graph_stats.begin(), b->graph_stats.end(), stats);
  if (!same) {
    int rc = upload_runs(b, stats, 0.0);
    if (rc) return rc;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (!b->cap_stream) BTRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    BTRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue(b, stats, b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bcuda(e != cudaSuccess ? e : e2, "batch graph capture");
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(e, "cudaGraphInstantiate");
    b->graph_stats.assign(stats, stats + b->count);
  }
  BTRY(cudaGraphLaunch(b->exec, s));  // zeroes every stats buffer, runs the persistent items
  return run_hbm_nets(b, stats, s, 0.0);
} catch (const std::bad_alloc&) {
  return bfail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return bfail(EULER_ERR_CUDA, "unexpected error");
}

int euler_batch_info(const euler_batch* b, int32_t* hbm_networks, int64_t* hbm_min_units,
                     int32_t* critical_path, int32_t* block, int32_t* tile_shift, int32_t* hbm_block,
                     int32_t* graph_steps) {
  if (!b) return bfail(EULER_ERR_ARG, "batch is NULL");
  if (hbm_networks) *hbm_networks = (int32_t)b->hbm_nets.size();
  if (hbm_min_units) *hbm_min_units = b->hbm_min_units;
  if (critical_path) *critical_path = b->cp_factor > 0.0 ? 1 : 0;
  if (block) *block = b->block;
  if (tile_shift) *tile_shift = b->rt_shift;
  if (hbm_block) *hbm_block = b->hbm_block;
  if (graph_steps) *graph_steps = b->hbm_graph_steps;
  return EULER_OK;
}

int euler_batch_status(euler_batch* b, void* cuda_stream) {
  if (!b) return bfail(EULER_ERR_ARG, "batch is NULL");
  int first = EULER_OK;
  for (euler_net* h : b->nets) {
    const int rc = euler_net_status(h, cuda_stream);
    if (rc && !first) first = rc;
  }
  return first;
}

void euler_batch_destroy(euler_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->d_nets);
  cudaFree(b->d_runs);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_sacc);
  delete b;
}

int euler_net_batch_simulate(euler_net* const* nets, const euler_run* runs, int32_t count,
                             int64_t* const* stats, void* cuda_stream) try {
  euler_batch* b = nullptr;
  int rc = euler_batch_create(&b, nets, runs, count);
  if (rc) return rc;
  rc = euler_batch_run(b, stats, cuda_stream);
  const int st = euler_batch_status(b, cuda_stream);
  euler_batch_destroy(b);
  return rc ? rc : st;
} catch (const std::bad_alloc&) {
  return bfail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return bfail(EULER_ERR_CUDA, "unexpected error");
}

}  // extern "C"
