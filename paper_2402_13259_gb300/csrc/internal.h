// internal.h -- device table layout and launch entry points shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace eulernet {

// Immutable network tables on the device (uploaded once by euler_net_create).
struct NetTables {
  int32_t n;          // stations
  int32_t E;          // edges (CSR nnz)
  int32_t L;          // levels (longest-path depth + 1)
  int32_t max_level;  // stations in the widest level
  const int32_t* lvl_ptr;      // [L+1] offsets into lvl_station
  const int32_t* lvl_station;  // [n] stations ordered by (level, index)
  const int32_t* row_ptr;      // [n+1] CSR (routing P)
  const float4* qc;            // [E] BinomConst of each edge's conditional split probability
  const int32_t* in_ptr;       // [n+1] CSC offsets (edges into each station)
  const int32_t* in_edge;      // [E] edge ids into each station
  const int32_t* servers;      // [n] m_i
  const float* mu;             // [n] mu_i rounded to float
  const int32_t* N0;           // [n] or nullptr
  const int32_t* ex_col;       // [n] column of the station in the Lambda table, or -1
  int32_t n_ex;                // stations with external arrivals
  const int32_t* pos_level;    // [n] level of each position of the level order
  int32_t ring;                // routed-count ring slots of the slot schedules:
                               // max(2, largest level gap of an edge + 1)
};

// Per-call parameters.
struct RunParams {
  const float4* p0;  // [n] BinomConst of 1 - e^{-mu_i dt}
  const float* lam;  // [K][n_ex] per-step arrival means
  float h;           // dt rounded to float
  int32_t K;         // steps
  uint32_t key0, key1;
  int64_t R;          // replications in this call
  int64_t rep_begin;  // global index of local replication 0
  int32_t scheme;     // 0 backward, 1 forward
  int32_t tile_reps;  // replications per tile (power of two)
  int64_t num_tiles;
  int32_t cap;        // rejection-loop cap
  int64_t wait_limit; // polls of one inter-warp wait before it gives up (pipelined form)
  int32_t wait_sleep_ns; // pause between polls (pipelined form), 0 = none
  int32_t test_stall; // nonzero: no warp publishes progress (tests the timeout path)
  int32_t sacc_in_global;  // batch kernel: per-station sums in the global scratch slot
  const float* muh;      // [n] mu_i dt rounded to float (Eq. (1)/(2) departures)
  int32_t dep_mode;      // 0 exact (Algorithm 1), 1 Eq. (1), 2 Eq. (2)
  const int32_t* mtab;   // [K][n] servers per step (staffing schedule), or nullptr
  // likelihood-ratio gradients (persistent form, GRAD kernels only)
  const float* p0f;   // [n] p0 as the sampler uses it
  const float* dlam;  // [K][n_ex][3] dLambda/d(a, b, phase)
  double* scores;     // [R][n+3] per-replication scores out
  int64_t* stats;     // output, see eulernet.h
  unsigned* err;      // latched error bits
  int32_t tau0 = 0;   // the run covers steps tau0+1 .. K (HBM form; a resumed run)
  uint32_t rk[20] = {};  // Philox round keys of (key0, key1), see set_round_keys
};

// The Philox round keys of (key0, key1) (key0 + r W0 for r < 10, then
// key1 + r W1), read by the kernels from their parameter space.
inline void set_round_keys(uint32_t* rk, uint32_t key0, uint32_t key1) {
  for (int r = 0; r < 10; ++r) {
    rk[r] = key0 + (uint32_t)r * 0x9E3779B9u;
    rk[10 + r] = key1 + (uint32_t)r * 0xBB67AE85u;
  }
}

// Shared-memory bytes of the persistent kernel for a tile of `tile_reps`
// with `ring` slots of routed counts (NetTables::ring for the slot schedules
// of tile_body, 1 for the step-by-step schedule).
int64_t persistent_smem_bytes(int32_t n, int32_t E, int32_t ring, int32_t tile_reps);

// Batched form: one persistent launch over (network, tile) work items.
cudaError_t batch_occupancy(int block, int smem, int* blocks_per_sm);
cudaError_t launch_batch(int scheme, bool ext, const NetTables* nets, const RunParams* runs, const int2* items,
                         int num_items, int* next_item, long long* sacc_scratch,
                         int64_t sacc_slot_len, int grid, int block, int smem, cudaStream_t s);

// Gradient form of the persistent kernel (scores into p.scores) and the
// fixed-order reduction of L_m(r) S_r over replications.
int64_t grad_smem_extra(int32_t n, int32_t n_ex, int32_t tile_reps);
cudaError_t grad_occupancy(int scheme, int block, int smem, int* blocks_per_sm);
cudaError_t launch_persistent_grad(const NetTables& t, const RunParams& p, int grid, int block,
                                   int smem, cudaStream_t s);
cudaError_t launch_grad_reduce(int32_t n, int64_t R, double dt, const int64_t* stats,
                               const double* scores, double* partial, double* grad, double* value,
                               double* grad_var, bool center, cudaStream_t s);

// out[k] = (b[k] + f[k]) / 2 in double.
cudaError_t launch_average(const int64_t* b, const int64_t* f, double* out, int64_t len,
                           cudaStream_t s);

// Launch the persistent shared-memory kernel.
cudaError_t launch_persistent(const NetTables& t, const RunParams& p, int grid, int block,
                              int smem, cudaStream_t s);

// Blocks of `block` threads with `smem` bytes that fit on one SM.
cudaError_t persistent_occupancy(int scheme, int block, int smem, int* blocks_per_sm);

// Level-pipelined form: W warps per 32-replication tile, warp w owns the
// level-ordered station slice lvl_station[wbeg[w] .. wbeg[w+1]); prod[w] and
// cons[w] are the bit masks of the warps it receives routed customers from and
// sends them to.
struct PipePlan {
  int32_t W;
  int32_t wbeg[33];
  uint32_t prod[32];
  uint32_t cons[32];
};
int64_t pipeline_smem_bytes(int32_t n, int32_t E);
cudaError_t pipeline_occupancy(int scheme, int block, int smem, int* blocks_per_sm);
cudaError_t launch_pipeline(const NetTables& t, const RunParams& p, const PipePlan& pp, int grid,
                            int smem, cudaStream_t s);

// HBM-state form: per-step kernels over state in global memory.
struct HbmState {
  int32_t* N;      // [n][R] station-major, replication-fastest
  int32_t* Redge;  // [max(depth, 2)][E][R]: routed counts of step tau in ring slot tau % depth
                   // (forward skewed) or tau % 2 (backward fused)
  int64_t* racc;   // [R][4] per-replication partial sums
  int32_t* tau;    // device step (or skewed-slot) counter, 1-based
  int64_t ld;      // leading dimension (>= R, multiple of 4)
  const int32_t* pos_level = nullptr;  // [n] level of lvl_station[k] (skewed forward only)
  int32_t depth = 1;                   // ring slots of Redge: max level gap of an edge + 1
  double* mu_acc = nullptr;            // gradients: [n][ld] score sums in mu_i, step order
  double* th_acc = nullptr;            // gradients: [n_ex][3][ld] score sums in (a, b, phase)
  // sojourn times (Algorithm 4): tagged customers c < S of every replication
  unsigned long long* cloc = nullptr;  // [S][ld] station << 32 | due step << 1 | setup pending
  int32_t* cpos = nullptr;             // [S][ld] > 0 waiting position, 0 in service
  int32_t* csteps = nullptr;           // [S][ld] steps accounted
  const int32_t* col = nullptr;        // [E] destination station of each edge
  int32_t S = 0;
  // checkpoint / resume: N_tau0 in and N_K out, [n][state_ld] (replication
  // fastest, this chunk's replications from column state_r0), or nullptr
  const int32_t* state_in = nullptr;
  int32_t* state_out = nullptr;
  int64_t state_ld = 0, state_r0 = 0;
  // Philox round keys of the run's seed (see PhiloxStream), read from the
  // kernel's parameter space
  uint32_t rk[20] = {};
};

inline void set_round_keys(HbmState& hs, uint32_t key0, uint32_t key1) { set_round_keys(hs.rk, key0, key1); }

// What the HBM form's per-step kernels compute besides the step.
enum HbmMode { kHbmPlain = 0, kHbmGrad = 1, kHbmSojourn = 2 };
int64_t hbm_smem_bytes(int32_t n, int32_t tile_reps);
cudaError_t launch_hbm_init(const NetTables& t, const RunParams& p, const HbmState& hs,
                            cudaStream_t s);
// One step's kernels (backward: 2 phases; forward: one per level), then the
// step counter advance.  Safe to capture in a CUDA graph.
cudaError_t launch_hbm_step(const NetTables& t, const RunParams& p, const HbmState& hs, int block,
                            const int32_t* lvl_ptr_host, cudaStream_t s);
// One captured slot of the HBM form at device counter + koff: backward, the
// gather of step tau - 1 fused with the draws of step tau (slots 1 .. K+1);
// forward, skewed slot tau (every station i runs its step tau - level(i) when
// that lies in 1..K).  Does not advance the counter.
cudaError_t launch_hbm_slot(const NetTables& t, const RunParams& p, const HbmState& hs, int block,
                            int32_t koff, int mode, cudaStream_t s);
// Sojourn times in the HBM form: customers enter `station` in step tau0
// (setup pending); finish writes out[r][c] (steps, or minus them if censored).
cudaError_t launch_hbm_sojourn_init(const RunParams& p, const HbmState& hs, int32_t station,
                                    int32_t tau0, cudaStream_t s);
cudaError_t launch_hbm_sojourn_finish(const RunParams& p, const HbmState& hs, int32_t* out,
                                      cudaStream_t s);
// Gradients in the HBM form: p.scores[r][c] from the score sums of hs.
cudaError_t launch_hbm_scores(const NetTables& t, const RunParams& p, const HbmState& hs,
                              cudaStream_t s);
cudaError_t launch_hbm_advance(const HbmState& hs, int32_t by, cudaStream_t s);
cudaError_t launch_hbm_finish(const NetTables& t, const RunParams& p, const HbmState& hs,
                              int64_t R_total, int64_t r0, cudaStream_t s);

}  // namespace eulernet
