// handle.h -- the library's network handle (private; shared by the host
// translation units, not part of the public ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/eulernet.h"
#include "internal.h"

struct euler_net {
  int32_t n = 0, E = 0, L = 0, max_level = 0, n_ex = 0;
  std::vector<int32_t> row_ptr, col, servers, lvl_ptr, lvl_station, ex_col, N0;
  std::vector<int32_t> ex_station;  // station of each column of the arrival-mean table
  uint64_t uid = 0;                 // unique per handle in this process
  uint64_t tables_gen = 0;          // bumped whenever the per-step tables' inputs change
  std::vector<double> prob, mu;
  int32_t arr_kind = EULER_ARR_NONE;
  std::vector<double> w, table;
  double a = 0, b = 0, period = 1, phase = 0, tab_dt = 1;
  int32_t table_len = 0;

  int device = 0, sm_count = 0, smem_optin = 0;
  int32_t *d_lvl_ptr = nullptr, *d_lvl_station = nullptr, *d_row_ptr = nullptr, *d_in_ptr = nullptr,
          *d_in_edge = nullptr, *d_servers = nullptr, *d_N0 = nullptr, *d_ex_col = nullptr;
  float4* d_qc = nullptr;
  float* d_mu = nullptr;
  unsigned* d_err = nullptr;

  // staffing schedule (host copy) and its per-step table
  std::vector<int32_t> sv_table;
  int32_t sv_len = 0;
  double sv_dt = 1.0;
  int32_t* d_mtab = nullptr;
  size_t mtab_cap = 0;
  float* d_muh = nullptr;

  // external arrival means of steps win_lo .. win_hi multiplied by win_factor
  // (a perturbation of the coupled gradient; off when win_hi < win_lo)
  int64_t win_lo = 1, win_hi = 0;
  double win_factor = 1.0;

  // per-(dt, T) tables of the last call
  double c_dt = -1.0, c_T = -1.0;
  int32_t c_K = 0;
  float4* d_p0 = nullptr;
  float* d_lam = nullptr;
  size_t lam_cap = 0;

  // likelihood-ratio gradient tables of the last (dt, T) and scratch
  double g_dt = -1.0, g_T = -1.0;
  float* d_p0f = nullptr;
  float* d_dlam = nullptr;
  size_t dlam_cap = 0;
  int64_t* d_gstats = nullptr;
  size_t gstats_cap = 0;
  double* d_gscores = nullptr;
  size_t gscores_cap = 0;
  double* d_gpartial = nullptr;
  size_t gpartial_cap = 0;
  double* d_gmu = nullptr;  // HBM-form gradients: score sums [n][ld]
  size_t gmu_cap = 0;
  double* d_gth = nullptr;  // and [n_ex][3][ld]
  size_t gth_cap = 0;
  unsigned long long* d_cloc = nullptr;  // HBM-form sojourn times: customer state
  int32_t* d_cpos = nullptr;
  int32_t* d_csteps = nullptr;
  size_t cust_cap = 0;

  // scratch of the average scheme
  int64_t* d_avg_b = nullptr;
  int64_t* d_avg_f = nullptr;
  size_t avg_cap = 0;

  // sojourn-time sampler: edge destinations and a statistics scratch
  int32_t* d_col = nullptr;
  int64_t* d_sstats = nullptr;
  size_t sstats_cap = 0;
  // HBM-form state; Redge holds hbm_depth ring slots (skewed forward scheme)
  int32_t *d_N = nullptr, *d_Redge = nullptr, *d_tau = nullptr, *d_pos_level = nullptr;
  int32_t hbm_depth = 0;
  int64_t* d_racc = nullptr;
  int64_t hbm_cap_ld = 0, hbm_cap_R = 0;
  cudaStream_t cap_stream = nullptr;

  int64_t opt[13] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
  int64_t h2d_bytes = 0;  // host-to-device bytes copied by this handle so far

  // The per-step tables depend on mu, the staffing schedule and the arrival
  // window: after a change they are rebuilt on the next call.
  void invalidate_step_tables() {
    c_dt = c_T = -1.0;
    ++tables_gen;
  }

  int32_t dep_mode() const { return opt[EULER_OPT_DEPARTURE] > 0 ? (int32_t)opt[EULER_OPT_DEPARTURE] : 0; }
  const int32_t* mtab() const { return sv_len > 0 ? d_mtab : nullptr; }

  eulernet::NetTables tables() const {
    eulernet::NetTables t;
    t.n = n;
    t.E = E;
    t.L = L;
    t.max_level = max_level;
    t.lvl_ptr = d_lvl_ptr;
    t.lvl_station = d_lvl_station;
    t.row_ptr = d_row_ptr;
    t.qc = d_qc;
    t.in_ptr = d_in_ptr;
    t.in_edge = d_in_edge;
    t.servers = d_servers;
    t.mu = d_mu;
    t.N0 = N0.empty() ? nullptr : d_N0;
    t.ex_col = d_ex_col;
    t.n_ex = n_ex;
    t.pos_level = d_pos_level;
    t.ring = hbm_depth > 2 ? hbm_depth : 2;
    return t;
  }
};

namespace eulernet {
// Units per step (n R) from which the planner takes the HBM form, and its
// default threads per block.
constexpr int64_t kHbmMinUnitsPerStep = int64_t(1) << 18;
constexpr int kHbmBlock = 256;
// Bytes of HBM-form state per replication chunk, so that a chunk stays in L2.
constexpr int64_t kHbmL2Budget = int64_t(64) << 20;

// What an HBM-form run computes besides the statistics (see HbmMode).
struct HbmExtra {
  int mode = kHbmPlain;
  double* mu_acc = nullptr;            // gradients: score sums, zeroed by the run
  double* th_acc = nullptr;
  unsigned long long* cloc = nullptr;  // sojourn times: customer state [S][ld]
  int32_t* cpos = nullptr;
  int32_t* csteps = nullptr;
  const int32_t* col = nullptr;
  int32_t S = 0, station = 0, tau0 = 0;
  int32_t* out = nullptr;              // [R][S]
  const int32_t* state_in = nullptr;   // checkpoint N_{p.tau0}, [n][R], or nullptr (N0)
  int32_t* state_out = nullptr;        // N_K out, [n][R], or nullptr
  int graph_steps = 0;                 // slots per CUDA graph replay (0: the handle's option)
};

// One call in the HBM form: state set-up, the graph of per-step kernels
// replayed to the horizon, statistics (and scores / sojourn times) out.
int run_hbm_form(euler_net* h, const NetTables& t, const RunParams& p, int block, cudaStream_t s,
                 const HbmExtra& x);

// A plain simulation call in the HBM form (the per-step kernels; the batched
// form's large networks): tables made current for (dt, T), `block` threads
// per step kernel, `graph_steps` slots per graph replay (0: default), at most
// k_limit steps when k_limit > 0 (tuning runs).  `stats` must be zeroed by
// the caller, on stream s.
int simulate_hbm(euler_net* h, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
                 int64_t rep_begin, int64_t* stats, cudaStream_t s, int block, int graph_steps,
                 int64_t k_limit);

// Per-step mean of the external arrivals of station i over step tau: the
// exact integral of lambda_i over ((tau-1) dt, tau dt] (Sec. 2.1.1), in double.
double step_mean(const euler_net& h, int32_t i, int64_t tau, double dt);
// Set the message euler_net_last_error() returns on this thread.
void set_last_error(const char* msg);
// Make the handle's per-call tables (p0 constants, Lambda) current for
// (dt, T) on stream s; returns an EULER_* code.
int prepare_step_tables(euler_net* h, double dt, double T, cudaStream_t s);

// The per-step tables of a call with step dt, written into host buffers in
// ranges, so that every entry point computes them the same way:
//   p0[k], muh[k] for stations i0 + k (k < cnt): the constants of the x <= m
//     departure probability 1 - e^{-mu_i dt} (Lemma 1) and mu_i dt in float;
//   servers[k * n + i] for steps tau0 + k (k < cnt): the staffing schedule's
//     value at the step's start (needs a schedule);
//   lam[k] for the flat entries j0 + k (k < cnt) of the [K][n_ex] table of
//     external-arrival means (Sec. 2.1.1), the arrival window's factor applied.
void step_p0(const euler_net& h, double dt, int32_t i0, int32_t cnt, float4* p0, float* muh);
void step_servers(const euler_net& h, double dt, int64_t tau0, int64_t cnt, int32_t* servers);
void step_lam(const euler_net& h, double dt, int64_t j0, int64_t cnt, float* lam);
}  // namespace eulernet
