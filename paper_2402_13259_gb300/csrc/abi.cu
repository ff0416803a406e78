// abi.cu -- host side of the C ABI declared in include/eulernet.h.
//
// euler_net_create validates the network (Sec. 2.2: routing probabilities
// p_ij with exit probability 1 - sum_j p_ij, servers m_i, rates mu_i), orders
// stations into levels by longest path (the flow order the forward scheme of
// Algorithm 3 needs for a feedforward network), builds the reverse graph for
// the gather of internal arrivals (Sec. 2.2, A^in_i = sum_k R_ki) and the
// conditional split probabilities of the sequential-binomial multinomial, and
// uploads everything once.  euler_net_simulate computes the per-step arrival
// means (Sec. 2.1.1, the integral of lambda_i over each step) for its (dt, T),
// picks the launch form and runs it asynchronously.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/eulernet.h"
#include "handle.h"
#include "internal.h"
#include "sampling.cuh"

using namespace eulernet;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

void eulernet::set_last_error(const char* msg) { g_last_error = msg; }

namespace {

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? EULER_ERR_OOM : EULER_ERR_CUDA;
}

#define CUDA_TRY(expr)                              \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src, int64_t* counter) {
  *dst = nullptr;
  *counter += (int64_t)(src.size() * sizeof(T));
  const size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

// Per-step mean of the external arrivals: the exact integral of lambda_i over
// ((tau-1) dt, tau dt] (Sec. 2.1.1), in double.
double eulernet::step_mean(const euler_net& h, int32_t i, int64_t tau, double dt) {
  const double t0 = (double)(tau - 1) * dt;
  const double t1 = (double)tau * dt;
  if (h.arr_kind == EULER_ARR_SINUSOID) {
    const double om = 6.283185307179586 / h.period;
    const double lam =
        h.w[i] * h.a * ((t1 - t0) + h.b * (cos(om * t0 + h.phase) - cos(om * t1 + h.phase)) / om);
    return lam > 0.0 ? lam : 0.0;
  }
  if (h.arr_kind == EULER_ARR_TABLE) {
    const int32_t J = h.table_len, n = h.n;
    const double td = h.tab_dt;
    double total = 0.0;
    double a = t0;
    while (a < t1) {
      const int64_t j = (int64_t)floor(a / td);
      const double seg_end = (double)(j + 1) * td;
      double b = seg_end < t1 ? seg_end : t1;
      if (b <= a) b = t1;
      double la, lb;
      if (j >= J - 1) {
        la = lb = h.table[(int64_t)(J - 1) * n + i];
      } else {
        const double y0 = h.table[j * n + i], y1 = h.table[(j + 1) * n + i];
        const double ta = (double)j * td;
        la = y0 + (y1 - y0) * ((a - ta) / td);
        lb = y0 + (y1 - y0) * ((b - ta) / td);
      }
      total += (b - a) * (la + lb) * 0.5;
      a = b;
    }
    return total > 0.0 ? total : 0.0;
  }
  return 0.0;
}

void eulernet::step_p0(const euler_net& h, double dt, int32_t i0, int32_t cnt, float4* p0, float* muh) {
  for (int32_t k = 0; k < cnt; ++k) {
    const float y = (float)(h.mu[i0 + k] * dt);
    const BinomConst bc = binom_const(-fm::expm1(-y));
    p0[k] = make_float4(bc.c0, bc.q, bc.r, bc.lq);
    muh[k] = y;
  }
}

void eulernet::step_servers(const euler_net& h, double dt, int64_t tau0, int64_t cnt, int32_t* servers) {
  for (int64_t k = 0; k < cnt; ++k) {
    const int64_t tau = tau0 + k;
    int64_t j = (int64_t)floor((double)(tau - 1) * dt / h.sv_dt);
    if (j > h.sv_len - 1) j = h.sv_len - 1;
    std::copy(h.sv_table.begin() + j * h.n, h.sv_table.begin() + (j + 1) * h.n, servers + k * h.n);
  }
}

void eulernet::step_lam(const euler_net& h, double dt, int64_t j0, int64_t cnt, float* lam) {
  for (int64_t k = 0; k < cnt; ++k) {
    const int64_t j = j0 + k;
    const int64_t tau = j / h.n_ex + 1;
    const int32_t i = h.ex_station[j % h.n_ex];
    double L = step_mean(h, i, tau, dt);
    if (tau >= h.win_lo && tau <= h.win_hi) L = L * h.win_factor;
    lam[k] = (float)L;
  }
}

namespace {

int refresh_step_tables(euler_net* h, double dt, double T, cudaStream_t s) {
  const int64_t K = euler_num_steps(dt, T);
  if (h->c_dt == dt && h->c_T == T) return EULER_OK;
  std::vector<float4> p0(h->n);
  std::vector<float> muh(h->n);
  step_p0(*h, dt, 0, h->n, p0.data(), muh.data());
  if (h->sv_len > 0) {
    std::vector<int32_t> mt((size_t)K * h->n);
    step_servers(*h, dt, 1, K, mt.data());
    if (mt.size() > h->mtab_cap || !h->d_mtab) {
      cudaFree(h->d_mtab);
      h->d_mtab = nullptr;
      CUDA_TRY(cudaMalloc(&h->d_mtab, sizeof(int32_t) * mt.size()));
      h->mtab_cap = mt.size();
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_mtab, mt.data(), sizeof(int32_t) * mt.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    h->h2d_bytes += (int64_t)(sizeof(int32_t) * mt.size());
  }
  if (!h->d_muh) CUDA_TRY(cudaMalloc(&h->d_muh, sizeof(float) * (size_t)h->n));
  CUDA_TRY(cudaMemcpyAsync(h->d_muh, muh.data(), sizeof(float) * muh.size(), cudaMemcpyHostToDevice, s));
  h->h2d_bytes += (int64_t)(sizeof(float) * muh.size());
  std::vector<float> lam((size_t)K * std::max(h->n_ex, 1), 0.0f);
  if (h->n_ex > 0) step_lam(*h, dt, 0, K * h->n_ex, lam.data());
  if (!h->d_p0) CUDA_TRY(cudaMalloc(&h->d_p0, sizeof(float4) * (size_t)h->n));
  if (lam.size() > h->lam_cap) {
    if (h->d_lam) CUDA_TRY(cudaFree(h->d_lam));
    h->d_lam = nullptr;
    CUDA_TRY(cudaMalloc(&h->d_lam, sizeof(float) * lam.size()));
    h->lam_cap = lam.size();
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_p0, p0.data(), sizeof(float4) * p0.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_lam, lam.data(), sizeof(float) * lam.size(), cudaMemcpyHostToDevice, s));
  h->h2d_bytes += (int64_t)(sizeof(float4) * p0.size() + sizeof(float) * lam.size());
  CUDA_TRY(cudaStreamSynchronize(s));  // host staging buffers go out of scope
  h->c_dt = dt;
  h->c_T = T;
  h->c_K = (int32_t)K;
  return EULER_OK;
}

}  // namespace

int eulernet::prepare_step_tables(euler_net* h, double dt, double T, cudaStream_t s) {
  return refresh_step_tables(h, dt, T, s);
}

namespace {

struct Plan {
  int form = 1, tile_reps = 32, block = 32, grid = 1;
  int64_t smem = 0, num_tiles = 0;
  PipePlan pipe;
};

// Cut the level-ordered stations into W contiguous slices and record, per
// slice, which other slices it receives from and sends to.
bool make_pipe_plan(const euler_net* h, int W, PipePlan* pp) {
  const int32_t n = h->n;
  if (W < 1 || W > 32 || W > n) return false;
  pp->W = W;
  for (int w = 0; w <= W; ++w) pp->wbeg[w] = (int32_t)(((int64_t)w * n) / W);
  std::vector<int32_t> owner(n, 0);
  for (int w = 0; w < W; ++w)
    for (int32_t k = pp->wbeg[w]; k < pp->wbeg[w + 1]; ++k) owner[h->lvl_station[k]] = w;
  for (int w = 0; w < 32; ++w) pp->prod[w] = pp->cons[w] = 0u;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) {
      const int a = owner[i], b = owner[h->col[e]];
      if (a == b) continue;
      if (a > b) return false;  // cannot happen for level order
      pp->cons[a] |= 1u << b;
      pp->prod[b] |= 1u << a;
    }
  return true;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }


int make_plan(euler_net* h, int32_t scheme, int64_t R, Plan* pl) {
  const int64_t limit = h->smem_optin;
  const int forced_form = (int)h->opt[EULER_OPT_FORM];
  int Rt = -1;
  if (h->opt[EULER_OPT_TILE_REPS] > 0) {
    Rt = (int)h->opt[EULER_OPT_TILE_REPS];
    if (!is_pow2(Rt) || Rt > 512) return fail(EULER_ERR_ARG, "tile replications must be a power of two <= 512");
  } else {
    for (int cand = 32; cand >= 1; cand >>= 1)
      if (persistent_smem_bytes(h->n, h->E, h->tables().ring, cand) <= limit) {
        Rt = cand;
        break;
      }
  }
  if (forced_form == 3) {
    const int W = h->opt[EULER_OPT_PIPE_WARPS] > 0 ? (int)h->opt[EULER_OPT_PIPE_WARPS]
                                                   : (int)std::min<int64_t>(h->n, 16);
    const int64_t psmem = pipeline_smem_bytes(h->n, h->E);
    bool fits = W <= 16 && psmem <= limit && make_pipe_plan(h, W, &pl->pipe);
    int per_sm = 0;
    if (fits) {
      cudaError_t e = pipeline_occupancy(scheme, 32 * W, (int)psmem, &per_sm);
      if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
      fits = per_sm >= 1;
    }
    if (fits) {
      pl->form = 3;
      pl->tile_reps = 32;
      pl->block = 32 * W;
      pl->smem = psmem;
      pl->num_tiles = (R + 31) / 32;
      int64_t grid = (int64_t)per_sm * h->sm_count;
      if (h->opt[EULER_OPT_GRID] > 0) grid = h->opt[EULER_OPT_GRID];
      pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, pl->num_tiles));
      return EULER_OK;
    }
    if (forced_form == 3) return fail(EULER_ERR_TOO_LARGE, "pipelined form does not fit");
  }
  pl->form = (forced_form == 1 || forced_form == 2) ? forced_form : 1;
  // With enough units in one step the HBM form wins: its per-step kernels
  // balance the stations' uneven sampler work over the whole GPU, where the
  // persistent form waits at block barriers every phase (forward: every
  // level), and its state traffic (about 8 + 8 deg bytes per unit) stays far
  // below HBM bandwidth.  Below the threshold launch gaps dominate.
  if (forced_form <= 0 && (int64_t)h->n * R >= kHbmMinUnitsPerStep) pl->form = 2;
  if (pl->form == 1 && (Rt < 1 || persistent_smem_bytes(h->n, h->E, h->tables().ring, Rt) > limit)) {
    if (forced_form == 1) return fail(EULER_ERR_TOO_LARGE, "network tile does not fit in shared memory");
    pl->form = 2;
  }
  if (pl->form == 2) {
    pl->tile_reps = 32;
    pl->block = h->opt[EULER_OPT_BLOCK] > 0 ? (int)h->opt[EULER_OPT_BLOCK] : kHbmBlock;
    if (pl->block % 32 || pl->block > 256) return fail(EULER_ERR_ARG, "HBM-form block must be a multiple of 32 <= 256");
    pl->grid = 0;
    pl->smem = 0;
    pl->num_tiles = (R + 31) / 32;
    return EULER_OK;
  }
  pl->tile_reps = Rt;
  const int64_t m_max = scheme == EULER_BACKWARD ? h->n : h->max_level;
  const int quantum = Rt >= 32 ? 1 : 32 / Rt;  // groups per warp
  int block;
  if (h->opt[EULER_OPT_BLOCK] > 0) {
    block = (int)h->opt[EULER_OPT_BLOCK];
    if (block % 32 || block % Rt || block > 512) return fail(EULER_ERR_ARG, "block must be a multiple of 32 and of the tile, <= 512");
  } else {
    const int64_t gmax = std::max<int64_t>(512 / Rt, 1);
    const int64_t iters = (m_max + gmax - 1) / gmax;
    int64_t G = (m_max + iters - 1) / iters;
    G = (G + quantum - 1) / quantum * quantum;
    if (G * Rt > 512) G = 512 / Rt;
    block = (int)std::max<int64_t>(G * Rt, 32);
  }
  pl->block = block;
  pl->smem = persistent_smem_bytes(h->n, h->E, h->tables().ring, Rt);
  pl->num_tiles = (R + Rt - 1) / Rt;
  int per_sm = 0;
  cudaError_t e = persistent_occupancy(scheme, block, (int)pl->smem, &per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    if (forced_form == 1) return fail(EULER_ERR_TOO_LARGE, "persistent kernel cannot be resident");
    pl->form = 2;
    pl->tile_reps = 32;
    pl->block = kHbmBlock;
    pl->num_tiles = (R + 31) / 32;
    return EULER_OK;
  }
  int64_t grid = (int64_t)per_sm * h->sm_count;
  if (h->opt[EULER_OPT_GRID] > 0) grid = h->opt[EULER_OPT_GRID];
  pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, pl->num_tiles));
  return EULER_OK;
}

// Level of each station position of the level order, and the ring depth of
// the skewed forward scheme: the largest level gap of an edge, plus one.
int ensure_levels(euler_net* h) {
  if (h->d_pos_level) return EULER_OK;
  std::vector<int32_t> pos_level(h->n), level(h->n);
  for (int32_t j = 0; j < h->L; ++j)
    for (int32_t k = h->lvl_ptr[j]; k < h->lvl_ptr[j + 1]; ++k) {
      pos_level[k] = j;
      level[h->lvl_station[k]] = j;
    }
  int32_t gap = 0;
  for (int32_t i = 0; i < h->n; ++i)
    for (int32_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e)
      gap = std::max(gap, level[h->col[e]] - level[i]);
  CUDA_TRY(cudaMalloc(&h->d_pos_level, sizeof(int32_t) * (size_t)h->n));
  CUDA_TRY(cudaMemcpy(h->d_pos_level, pos_level.data(), sizeof(int32_t) * (size_t)h->n,
                      cudaMemcpyHostToDevice));
  h->h2d_bytes += (int64_t)sizeof(int32_t) * h->n;
  h->hbm_depth = gap + 1;
  return EULER_OK;
}

int ensure_hbm_state(euler_net* h, int64_t R) {
  int rc = ensure_levels(h);
  if (rc) return rc;
  const int64_t ld = (R + 3) / 4 * 4;
  if (ld <= h->hbm_cap_ld && R <= h->hbm_cap_R && h->d_N) return EULER_OK;
  cudaFree(h->d_N);
  cudaFree(h->d_Redge);
  cudaFree(h->d_racc);
  h->d_N = nullptr;
  h->d_Redge = nullptr;
  h->d_racc = nullptr;
  CUDA_TRY(cudaMalloc(&h->d_N, sizeof(int32_t) * (size_t)h->n * ld));
  CUDA_TRY(cudaMalloc(&h->d_Redge,
                      sizeof(int32_t) * (size_t)std::max(h->hbm_depth, 2) * std::max(h->E, 1) * ld));
  CUDA_TRY(cudaMalloc(&h->d_racc, sizeof(int64_t) * 4 * (size_t)std::max<int64_t>(R, 1)));
  if (!h->d_tau) CUDA_TRY(cudaMalloc(&h->d_tau, sizeof(int32_t)));
  h->hbm_cap_ld = ld;
  h->hbm_cap_R = R;
  return EULER_OK;
}

int64_t hbm_slots(const euler_net* h, int32_t scheme, int64_t K) {
  return scheme == EULER_BACKWARD ? K + 1 : K + h->L - 1;
}

}  // namespace

// The HBM form of one call: init, the graph of per-step kernels replayed to
// the horizon, finish.  Gradients: the kernels also sum the score terms into
// x.mu_acc / x.th_acc (zeroed here) and the scores go to p.scores.  Sojourn
// times: the customers start at x.station, step x.tau0, and their sojourns go
// to x.out.
int eulernet::run_hbm_form(euler_net* h, const NetTables& t, const RunParams& p, int block,
                           cudaStream_t s, const HbmExtra& x) {
  int rc = ensure_levels(h);
  if (rc) return rc;
  // Replications in chunks whose state (N, the routed-count ring, the
  // per-replication sums and the mode's extra sums) fits in about
  // kHbmL2Budget bytes of L2, whole horizon per chunk: counter-based keying
  // makes the results those of one pass.  A chunk keeps n x R >= 2^18 units
  // per step.
  const int64_t per_rep = 4 * ((int64_t)h->n + std::max(h->hbm_depth, 2) * (int64_t)h->E) + 32 +
                          (x.mode == kHbmGrad ? 8 * ((int64_t)h->n + 3 * (int64_t)std::max(h->n_ex, 1)) : 0) +
                          (x.mode == kHbmSojourn ? 16 * (int64_t)x.S : 0);
  int64_t Rc = h->opt[EULER_OPT_HBM_CHUNK] > 0
                   ? h->opt[EULER_OPT_HBM_CHUNK]
                   : std::max<int64_t>(kHbmL2Budget / per_rep, (kHbmMinUnitsPerStep + h->n - 1) / h->n);
  Rc = (Rc + 31) / 32 * 32;
  if (Rc > p.R) Rc = p.R;
  rc = ensure_hbm_state(h, Rc);
  if (rc) return rc;
  HbmState hs;
  hs.N = h->d_N;
  hs.Redge = h->d_Redge;
  hs.racc = h->d_racc;
  hs.tau = h->d_tau;
  hs.ld = h->hbm_cap_ld;
  hs.pos_level = h->d_pos_level;
  hs.depth = h->hbm_depth;
  hs.mu_acc = x.mu_acc;
  hs.th_acc = x.th_acc;
  hs.cloc = x.cloc;
  hs.cpos = x.cpos;
  hs.csteps = x.csteps;
  hs.col = x.col;
  hs.S = x.S;
  hs.state_in = x.state_in;
  hs.state_out = x.state_out;
  hs.state_ld = p.R;
  set_round_keys(hs, p.key0, p.key1);
  // backward: K + 1 fused slots; forward: K + L - 1 skewed slots (from
  // slot tau0 + 1 in a resumed run)
  const int64_t slots = hbm_slots(h, p.scheme, p.K) - p.tau0;
  const int64_t S = x.graph_steps > 0 ? std::min<int64_t>(x.graph_steps, std::max<int64_t>(slots, 1))
                   : h->opt[EULER_OPT_GRAPH_STEPS] > 0 ? h->opt[EULER_OPT_GRAPH_STEPS]
                                                        : std::min<int64_t>(std::max<int64_t>(slots, 1), 32);
  if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  for (int64_t r0 = 0; r0 < p.R; r0 += Rc) {
    RunParams pc = p;
    pc.R = std::min<int64_t>(Rc, p.R - r0);
    pc.rep_begin = p.rep_begin + r0;
    pc.num_tiles = (pc.R + 31) / 32;
    hs.state_r0 = r0;
    if (x.mode == kHbmGrad) {
      pc.scores = p.scores + r0 * ((int64_t)h->n + 3);
      CUDA_TRY(cudaMemsetAsync(x.mu_acc, 0, sizeof(double) * (size_t)h->n * hs.ld, s));
      CUDA_TRY(cudaMemsetAsync(x.th_acc, 0, sizeof(double) * (size_t)std::max(h->n_ex, 1) * 3 * hs.ld, s));
    }
    if (x.mode == kHbmSojourn) CUDA_TRY(launch_hbm_sojourn_init(pc, hs, x.station, x.tau0, s));
    CUDA_TRY(launch_hbm_init(t, pc, hs, s));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int64_t k = 0; k <= S; ++k) {
      cudaError_t e = k < S ? launch_hbm_slot(t, pc, hs, block, (int32_t)k, x.mode, h->cap_stream)
                            : launch_hbm_advance(hs, (int32_t)S, h->cap_stream);
      if (e != cudaSuccess) {
        cudaStreamEndCapture(h->cap_stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e, "hbm step capture");
      }
    }
    CUDA_TRY(cudaStreamEndCapture(h->cap_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    const int64_t replays = slots > 0 ? (slots + S - 1) / S : 0;
    for (int64_t k = 0; k < replays && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    CUDA_TRY(launch_hbm_finish(t, pc, hs, p.R, r0, s));
    if (x.mode == kHbmGrad) CUDA_TRY(launch_hbm_scores(t, pc, hs, s));
    if (x.mode == kHbmSojourn) CUDA_TRY(launch_hbm_sojourn_finish(pc, hs, x.out + r0 * x.S, s));
  }
  return EULER_OK;
}

namespace {

int validate_net(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* prob,
                 const int32_t* servers, const double* mu, const euler_arrivals* arr,
                 const int32_t* N0) {
  if (n <= 0 || n >= (1 << 24)) return fail(EULER_ERR_ARG, "n must be in [1, 2^24)");
  if (!row_ptr || !servers || !mu) return fail(EULER_ERR_ARG, "row_ptr, servers and mu are required");
  if (row_ptr[0] != 0) return fail(EULER_ERR_ARG, "row_ptr[0] must be 0");
  for (int32_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return fail(EULER_ERR_ARG, "row_ptr must be non-decreasing");
    if (row_ptr[i + 1] >= (1 << 30)) return fail(EULER_ERR_TOO_LARGE, "too many edges");
    if (servers[i] < 1) return fail(EULER_ERR_ARG, "servers must be >= 1");
    if (!(mu[i] > 0.0) || !std::isfinite(mu[i])) return fail(EULER_ERR_ARG, "mu must be finite and > 0");
    if (N0 && (N0[i] < 0 || N0[i] > kStateLimit)) return fail(EULER_ERR_ARG, "N0 out of range");
  }
  const int32_t E = row_ptr[n];
  if (E > 0 && (!col || !prob)) return fail(EULER_ERR_ARG, "col and prob are required");
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (col[e] < 0 || col[e] >= n) return fail(EULER_ERR_ARG, "edge destination out of range");
      if (col[e] == i) return fail(EULER_ERR_NOT_FEEDFORWARD, "self loop");
      if (!(prob[e] >= 0.0 && prob[e] <= 1.0)) return fail(EULER_ERR_ARG, "edge probability outside [0,1]");
      s += prob[e];
    }
    if (s > 1.0 + 1e-12) return fail(EULER_ERR_ARG, "routing row sum exceeds 1");
  }
  if (arr && arr->kind == EULER_ARR_SINUSOID) {
    if (!arr->w || !(arr->period > 0.0) || !std::isfinite(arr->a) || !std::isfinite(arr->b))
      return fail(EULER_ERR_ARG, "bad sinusoid arrival parameters");
    for (int32_t i = 0; i < n; ++i)
      if (!(arr->w[i] >= 0.0) || !std::isfinite(arr->w[i])) return fail(EULER_ERR_ARG, "arrival weights must be finite and >= 0");
  } else if (arr && arr->kind == EULER_ARR_TABLE) {
    if (!arr->table || arr->table_len < 1 || !(arr->tab_dt > 0.0)) return fail(EULER_ERR_ARG, "bad arrival table");
    for (int64_t k = 0; k < (int64_t)arr->table_len * n; ++k)
      if (!(arr->table[k] >= 0.0) || !std::isfinite(arr->table[k])) return fail(EULER_ERR_ARG, "arrival table must be finite and >= 0");
  } else if (arr && arr->kind != EULER_ARR_NONE) {
    return fail(EULER_ERR_ARG, "unknown arrival kind");
  }
  return EULER_OK;
}

}  // namespace

extern "C" {

int64_t euler_num_steps(double dt, double T) {
  const double k = ceil(T / dt - 1e-9);
  return k < 1.0 ? 1 : (int64_t)k;
}

int64_t euler_stats_len(int32_t n, int64_t replications) { return 6 * (int64_t)n + 4 * replications; }

const char* euler_net_last_error(void) { return g_last_error.c_str(); }

void euler_net_destroy(euler_net* h) {
  if (!h) return;
  cudaFree(h->d_lvl_ptr);
  cudaFree(h->d_lvl_station);
  cudaFree(h->d_row_ptr);
  cudaFree(h->d_in_ptr);
  cudaFree(h->d_in_edge);
  cudaFree(h->d_servers);
  cudaFree(h->d_N0);
  cudaFree(h->d_ex_col);
  cudaFree(h->d_qc);
  cudaFree(h->d_mu);
  cudaFree(h->d_err);
  cudaFree(h->d_p0);
  cudaFree(h->d_lam);
  cudaFree(h->d_N);
  cudaFree(h->d_Redge);
  cudaFree(h->d_racc);
  cudaFree(h->d_tau);
  cudaFree(h->d_p0f);
  cudaFree(h->d_dlam);
  cudaFree(h->d_gstats);
  cudaFree(h->d_gscores);
  cudaFree(h->d_gpartial);
  cudaFree(h->d_avg_b);
  cudaFree(h->d_avg_f);
  cudaFree(h->d_mtab);
  cudaFree(h->d_muh);
  cudaFree(h->d_col);
  cudaFree(h->d_sstats);
  cudaFree(h->d_pos_level);
  cudaFree(h->d_gmu);
  cudaFree(h->d_gth);
  cudaFree(h->d_cloc);
  cudaFree(h->d_cpos);
  cudaFree(h->d_csteps);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

int euler_net_create(euler_net** out, int32_t n, const int32_t* row_ptr, const int32_t* col,
                     const double* prob, const int32_t* servers, const double* mu,
                     const euler_arrivals* arrivals, const int32_t* N0) try {
  if (!out) return fail(EULER_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate_net(n, row_ptr, col, prob, servers, mu, arrivals, N0);
  if (rc) return rc;
  euler_net* h = new euler_net();
  h->n = n;
  h->E = row_ptr[n];
  h->row_ptr.assign(row_ptr, row_ptr + n + 1);
  h->col.assign(col ? col : row_ptr, col ? col + h->E : row_ptr);
  h->prob.assign(prob ? prob : mu, prob ? prob + h->E : mu);
  h->servers.assign(servers, servers + n);
  h->mu.assign(mu, mu + n);
  if (N0) h->N0.assign(N0, N0 + n);
  if (arrivals) {
    h->arr_kind = arrivals->kind;
    if (arrivals->kind == EULER_ARR_SINUSOID) {
      h->w.assign(arrivals->w, arrivals->w + n);
      h->a = arrivals->a;
      h->b = arrivals->b;
      h->period = arrivals->period;
      h->phase = arrivals->phase;
    } else if (arrivals->kind == EULER_ARR_TABLE) {
      h->table.assign(arrivals->table, arrivals->table + (int64_t)arrivals->table_len * n);
      h->table_len = arrivals->table_len;
      h->tab_dt = arrivals->tab_dt;
    }
  }

  // levels by longest path, via Kahn's order; a leftover station means a cycle
  std::vector<int32_t> indeg(n, 0), level(n, 0), ready;
  for (int32_t e = 0; e < h->E; ++e) indeg[h->col[e]]++;
  for (int32_t i = 0; i < n; ++i)
    if (indeg[i] == 0) ready.push_back(i);
  size_t head = 0;
  while (head < ready.size()) {
    const int32_t i = ready[head++];
    for (int32_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) {
      const int32_t j = h->col[e];
      level[j] = std::max(level[j], level[i] + 1);
      if (--indeg[j] == 0) ready.push_back(j);
    }
  }
  if ((int32_t)ready.size() != n) {
    delete h;
    return fail(EULER_ERR_NOT_FEEDFORWARD, "routing graph has a cycle");
  }
  h->L = 1 + *std::max_element(level.begin(), level.end());
  h->lvl_ptr.assign(h->L + 1, 0);
  for (int32_t i = 0; i < n; ++i) h->lvl_ptr[level[i] + 1]++;
  for (int32_t j = 0; j < h->L; ++j) h->lvl_ptr[j + 1] += h->lvl_ptr[j];
  h->lvl_station.assign(n, 0);
  {
    std::vector<int32_t> fill(h->lvl_ptr.begin(), h->lvl_ptr.end() - 1);
    for (int32_t i = 0; i < n; ++i) h->lvl_station[fill[level[i]]++] = i;
  }
  h->max_level = 0;
  for (int32_t j = 0; j < h->L; ++j) h->max_level = std::max(h->max_level, h->lvl_ptr[j + 1] - h->lvl_ptr[j]);

  // conditional split probabilities qc_e = p_e / (p_exit + sum_{e' >= e} p_e')
  std::vector<float> qc(std::max(h->E, 1), 0.0f);  // conditional split probabilities
  for (int32_t i = 0; i < n; ++i) {
    const int32_t e0 = h->row_ptr[i], e1 = h->row_ptr[i + 1];
    double rowsum = 0.0;
    for (int32_t e = e0; e < e1; ++e) rowsum += h->prob[e];
    double pexit = 1.0 - rowsum;
    if (pexit < 1e-12) pexit = 0.0;
    double suffix = pexit;
    for (int32_t e = e1 - 1; e >= e0; --e) {
      suffix += h->prob[e];
      double q = suffix > 0.0 ? h->prob[e] / suffix : 0.0;
      q = std::min(1.0, std::max(0.0, q));
      qc[e] = (float)q;
    }
  }
  // reverse graph
  std::vector<int32_t> in_ptr(n + 1, 0), in_edge(std::max(h->E, 1), 0);
  for (int32_t e = 0; e < h->E; ++e) in_ptr[h->col[e] + 1]++;
  for (int32_t i = 0; i < n; ++i) in_ptr[i + 1] += in_ptr[i];
  {
    std::vector<int32_t> fill(in_ptr.begin(), in_ptr.end() - 1);
    for (int32_t i = 0; i < n; ++i)
      for (int32_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) in_edge[fill[h->col[e]]++] = e;
  }
  // stations with external arrivals
  h->ex_col.assign(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    bool ext = false;
    if (h->arr_kind == EULER_ARR_SINUSOID) ext = h->w[i] != 0.0 && h->a != 0.0;
    if (h->arr_kind == EULER_ARR_TABLE)
      for (int32_t j = 0; j < h->table_len && !ext; ++j) ext = h->table[(int64_t)j * n + i] != 0.0;
    if (ext) {
      h->ex_col[i] = h->n_ex++;
      h->ex_station.push_back(i);
    }
  }
  {
    static std::atomic<uint64_t> next_uid{1};
    h->uid = next_uid.fetch_add(1);
  }
  std::vector<float4> qc_const(qc.size());
  for (size_t e = 0; e < qc.size(); ++e) {
    const BinomConst bc = binom_const(qc[e]);
    qc_const[e] = make_float4(bc.c0, bc.q, bc.r, bc.lq);
  }
  std::vector<float> mu_f(n);
  for (int32_t i = 0; i < n; ++i) mu_f[i] = (float)h->mu[i];

  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e == cudaSuccess) e = upload(&h->d_lvl_ptr, h->lvl_ptr, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_lvl_station, h->lvl_station, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_row_ptr, h->row_ptr, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_in_ptr, in_ptr, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_in_edge, in_edge, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_servers, h->servers, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_N0, h->N0, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_ex_col, h->ex_col, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_qc, qc_const, &h->h2d_bytes);
  if (e == cudaSuccess) e = upload(&h->d_mu, mu_f, &h->h2d_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    euler_net_destroy(h);
    return cuda_fail(e, "euler_net_create upload");
  }
  rc = ensure_levels(h);  // the slot schedules' levels and ring depth
  if (rc) {
    euler_net_destroy(h);
    return rc;
  }
  *out = h;
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

int64_t euler_net_h2d_bytes(const euler_net* h) { return h ? h->h2d_bytes : -1; }

int euler_net_set_servers_schedule(euler_net* h, const int32_t* table, int32_t len, double tab_dt) try {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  if (!table || len <= 0) {
    h->sv_table.clear();
    h->sv_len = 0;
  } else {
    if (!(tab_dt > 0.0) || !std::isfinite(tab_dt)) return fail(EULER_ERR_ARG, "schedule step must be finite and > 0");
    for (int64_t k = 0; k < (int64_t)len * h->n; ++k)
      if (table[k] < 1) return fail(EULER_ERR_ARG, "scheduled servers must be >= 1");
    h->sv_table.assign(table, table + (int64_t)len * h->n);
    h->sv_len = len;
    h->sv_dt = tab_dt;
  }
  h->invalidate_step_tables();  // rebuild the per-step tables on the next call
  h->g_dt = h->g_T = -1.0;
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

int euler_net_set_option(euler_net* h, int32_t option, int64_t value) {
  if (!h || option < 0 || option > EULER_OPT_HBM_CHUNK) return fail(EULER_ERR_ARG, "bad option");
  h->opt[option] = value < 0 ? -1 : value;
  return EULER_OK;
}

int euler_net_plan(euler_net* h, int32_t scheme, int64_t R, int32_t* form, int32_t* tile_reps,
                   int32_t* block, int32_t* grid, int32_t* smem_bytes) try {
  if (!h || R < 1) return fail(EULER_ERR_ARG, "bad plan arguments");
  Plan pl;
  int rc = make_plan(h, scheme, R, &pl);
  if (rc) return rc;
  if (form) *form = pl.form;
  if (tile_reps) *tile_reps = pl.tile_reps;
  if (block) *block = pl.block;
  if (grid) *grid = pl.grid;
  if (smem_bytes) *smem_bytes = (int32_t)pl.smem;
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

}  // extern "C"

namespace {

// The run parameters of a plain simulation call (tables current for dt).
RunParams simulate_params(const euler_net* h, int32_t scheme, double dt, int64_t K, int64_t R, uint64_t seed,
                          int64_t rep_begin, int64_t* stats, int32_t tile_reps, int64_t num_tiles) {
  RunParams p;
  p.p0 = h->d_p0;
  p.lam = h->d_lam;
  p.h = (float)dt;
  p.K = (int32_t)K;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  set_round_keys(p.rk, p.key0, p.key1);
  p.R = R;
  p.rep_begin = rep_begin;
  p.scheme = scheme;
  p.tile_reps = tile_reps;
  p.num_tiles = num_tiles;
  p.cap = h->opt[EULER_OPT_SAMPLER_CAP] > 0 ? (int32_t)h->opt[EULER_OPT_SAMPLER_CAP] : 1000;
  p.stats = stats;
  p.err = h->d_err;
  p.wait_limit = h->opt[EULER_OPT_WAIT_LIMIT] > 0 ? h->opt[EULER_OPT_WAIT_LIMIT] : (int64_t)1 << 25;
  p.test_stall = h->opt[EULER_OPT_TEST_STALL] > 0 ? 1 : 0;
  p.wait_sleep_ns = h->opt[EULER_OPT_WAIT_SLEEP] >= 0 ? (int32_t)std::min<int64_t>(h->opt[EULER_OPT_WAIT_SLEEP], 1000000) : 64;
  p.muh = h->d_muh;
  p.dep_mode = h->dep_mode();
  p.mtab = h->mtab();
  return p;
}

}  // namespace

int eulernet::simulate_hbm(euler_net* h, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
                           int64_t rep_begin, int64_t* stats, cudaStream_t s, int block, int graph_steps,
                           int64_t k_limit) {
  int rc = refresh_step_tables(h, dt, T, s);
  if (rc) return rc;
  int64_t K = euler_num_steps(dt, T);
  if (k_limit > 0 && K > k_limit) K = k_limit;
  if (R == 0) return EULER_OK;
  const RunParams p = simulate_params(h, scheme, dt, K, R, seed, rep_begin, stats, 32, (R + 31) / 32);
  HbmExtra x;
  x.graph_steps = graph_steps;
  return run_hbm_form(h, h->tables(), p, block, s, x);
}

extern "C" {

int euler_net_simulate(euler_net* h, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
                       int64_t rep_begin, int64_t* stats, void* stream) try {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  if (scheme != EULER_BACKWARD && scheme != EULER_FORWARD) return fail(EULER_ERR_ARG, "unknown scheme");
  if (!(dt > 0.0) || !(T > 0.0) || !std::isfinite(dt) || !std::isfinite(T)) return fail(EULER_ERR_ARG, "dt and T must be finite and > 0");
  if (R < 0 || rep_begin < 0 || !stats) return fail(EULER_ERR_ARG, "bad replications, rep_begin or stats");
  if (rep_begin + R > (int64_t)1 << 32) return fail(EULER_ERR_TOO_LARGE, "replication index beyond 2^32");
  const int64_t K = euler_num_steps(dt, T);
  if (K >= (1 << 24)) return fail(EULER_ERR_TOO_LARGE, "too many steps (T/dt >= 2^24)");
  if (h->n_ex > 0 && K * (int64_t)h->n_ex > ((int64_t)1 << 31)) return fail(EULER_ERR_TOO_LARGE, "arrival table too large");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemsetAsync(stats, 0, sizeof(int64_t) * (size_t)euler_stats_len(h->n, R), s));
  if (R == 0) return EULER_OK;
  int rc = refresh_step_tables(h, dt, T, s);
  if (rc) return rc;
  Plan pl;
  rc = make_plan(h, scheme, R, &pl);
  if (rc) return rc;
  const RunParams p = simulate_params(h, scheme, dt, K, R, seed, rep_begin, stats, pl.tile_reps, pl.num_tiles);
  const NetTables t = h->tables();
  if (pl.form == 3) {
    cudaError_t e = launch_pipeline(t, p, pl.pipe, pl.grid, (int)pl.smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "pipelined kernel launch");
    return EULER_OK;
  }
  if (pl.form == 1) {
    cudaError_t e = launch_persistent(t, p, pl.grid, pl.block, (int)pl.smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
    return EULER_OK;
  }
  return run_hbm_form(h, t, p, pl.block, s, HbmExtra());
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

}  // extern "C"

namespace {

// dLambda/d(a, b, phase) of station i over step tau (sinusoid arrivals; zero
// for a table or where Lambda is clamped at zero), in double.
void step_mean_grad(const euler_net& h, int32_t i, int64_t tau, double dt, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (h.arr_kind != EULER_ARR_SINUSOID) return;
  if (!(step_mean(h, i, tau, dt) > 0.0)) return;
  const double t0 = (double)(tau - 1) * dt;
  const double t1 = (double)tau * dt;
  const double om = 6.283185307179586 / h.period;
  const double c0 = cos(om * t0 + h.phase), c1 = cos(om * t1 + h.phase);
  const double s0 = sin(om * t0 + h.phase), s1 = sin(om * t1 + h.phase);
  g[0] = h.w[i] * ((t1 - t0) + h.b * (c0 - c1) / om);
  g[1] = h.w[i] * h.a * ((c0 - c1) / om);
  g[2] = h.w[i] * h.a * h.b * ((s1 - s0) / om);
}

template <class T>
int grow(T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return EULER_OK;
  cudaFree(*p);
  *p = nullptr;
  CUDA_TRY(cudaMalloc(p, sizeof(T) * std::max<size_t>(need, 1)));
  *cap = need;
  return EULER_OK;
}

int refresh_grad_tables(euler_net* h, double dt, double T, cudaStream_t s) {
  if (h->g_dt == dt && h->g_T == T) return EULER_OK;
  const int64_t K = euler_num_steps(dt, T);
  std::vector<float> p0f(h->n);
  for (int32_t i = 0; i < h->n; ++i) p0f[i] = -fm::expm1(-(float)(h->mu[i] * dt));
  std::vector<float> dl((size_t)K * std::max(h->n_ex, 1) * 3, 0.0f);
  for (int32_t i = 0; i < h->n; ++i) {
    const int32_t c = h->ex_col[i];
    if (c < 0) continue;
    for (int64_t tau = 1; tau <= K; ++tau) {
      double g[3];
      step_mean_grad(*h, i, tau, dt, g);
      for (int k = 0; k < 3; ++k) dl[((size_t)(tau - 1) * h->n_ex + c) * 3 + k] = (float)g[k];
    }
  }
  if (!h->d_p0f) CUDA_TRY(cudaMalloc(&h->d_p0f, sizeof(float) * (size_t)h->n));
  int rc = grow(&h->d_dlam, &h->dlam_cap, dl.size());
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(h->d_p0f, p0f.data(), sizeof(float) * p0f.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_dlam, dl.data(), sizeof(float) * dl.size(), cudaMemcpyHostToDevice, s));
  h->h2d_bytes += (int64_t)(sizeof(float) * (p0f.size() + dl.size()));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->g_dt = dt;
  h->g_T = T;
  return EULER_OK;
}

}  // namespace

extern "C" {

int euler_net_grad(euler_net* h, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
                   int64_t rep_begin, double* grad, double* value, double* grad_var, double* scores,
                   int64_t* stats, void* stream) try {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  if (scheme != EULER_BACKWARD && scheme != EULER_FORWARD) return fail(EULER_ERR_ARG, "unknown scheme");
  if (!(dt > 0.0) || !(T > 0.0) || !std::isfinite(dt) || !std::isfinite(T)) return fail(EULER_ERR_ARG, "dt and T must be finite and > 0");
  if (R < 1 || rep_begin < 0 || !grad || !value) return fail(EULER_ERR_ARG, "bad replications, rep_begin, grad or value");
  if (h->dep_mode() != 0) return fail(EULER_ERR_ARG, "gradients need the exact departure sampler (EULER_OPT_DEPARTURE = 0)");
  if (rep_begin + R > (int64_t)1 << 32) return fail(EULER_ERR_TOO_LARGE, "replication index beyond 2^32");
  const int64_t K = euler_num_steps(dt, T);
  if (K >= (1 << 24)) return fail(EULER_ERR_TOO_LARGE, "too many steps (T/dt >= 2^24)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = refresh_step_tables(h, dt, T, s);
  if (rc) return rc;
  rc = refresh_grad_tables(h, dt, T, s);
  if (rc) return rc;
  const int64_t C = (int64_t)h->n + 3;
  if (!stats) {
    rc = grow(&h->d_gstats, &h->gstats_cap, (size_t)euler_stats_len(h->n, R));
    if (rc) return rc;
    stats = h->d_gstats;
  }
  if (!scores) {
    rc = grow(&h->d_gscores, &h->gscores_cap, (size_t)(R * C));
    if (rc) return rc;
    scores = h->d_gscores;
  }
  const int64_t nb = (R + 31) / 32;
  rc = grow(&h->d_gpartial, &h->gpartial_cap, (size_t)(4 * nb * C + 2 * nb));
  if (rc) return rc;
  // At scale the HBM form (score sums per station and replication in global
  // memory, the same step order) is faster, as for euler_net_simulate.
  const int forced = (int)h->opt[EULER_OPT_FORM];
  if (forced == 2 || (forced <= 0 && (int64_t)h->n * R >= kHbmMinUnitsPerStep)) {
    const int64_t ld = (R + 3) / 4 * 4;
    rc = grow(&h->d_gmu, &h->gmu_cap, (size_t)(h->n * ld));
    if (rc) return rc;
    rc = grow(&h->d_gth, &h->gth_cap, (size_t)(std::max(h->n_ex, 1) * 3 * ld));
    if (rc) return rc;
    RunParams p;
    std::memset(&p, 0, sizeof p);
    p.p0 = h->d_p0;
    p.lam = h->d_lam;
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
    p.err = h->d_err;
    p.wait_limit = (int64_t)1 << 25;
    p.p0f = h->d_p0f;
    p.dlam = h->d_dlam;
    p.scores = scores;
    p.muh = h->d_muh;
    p.dep_mode = 0;
    p.mtab = h->mtab();
    Plan pl;
    pl.form = 2;
    pl.block = h->opt[EULER_OPT_BLOCK] > 0 ? (int)h->opt[EULER_OPT_BLOCK] : kHbmBlock;
    if (pl.block % 32 || pl.block > 256) return fail(EULER_ERR_ARG, "HBM-form block must be a multiple of 32 <= 256");
    CUDA_TRY(cudaMemsetAsync(stats, 0, sizeof(int64_t) * (size_t)euler_stats_len(h->n, R), s));
    HbmExtra xg;
    xg.mode = kHbmGrad;
    xg.mu_acc = h->d_gmu;
    xg.th_acc = h->d_gth;
    rc = run_hbm_form(h, h->tables(), p, pl.block, s, xg);
    if (rc) return rc;
    cudaError_t e = launch_grad_reduce(h->n, R, dt, stats, scores, h->d_gpartial, grad, value, grad_var,
                                       h->opt[EULER_OPT_GRAD_CENTER] > 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
    return EULER_OK;
  }
  // tile: the largest power of two <= 32 whose state and score sums fit
  int Rt = 32;
  int64_t smem = 0;
  for (; Rt >= 1; Rt /= 2) {
    smem = persistent_smem_bytes(h->n, h->E, h->tables().ring, Rt) + grad_smem_extra(h->n, h->n_ex, Rt);
    if (smem <= h->smem_optin) break;
  }
  if (Rt < 1) return fail(EULER_ERR_TOO_LARGE, "gradient tile does not fit in shared memory");
  const int64_t m_max = scheme == EULER_BACKWARD ? h->n : h->max_level;
  const int quantum = Rt >= 32 ? 1 : 32 / Rt;
  const int64_t gmax = std::max<int64_t>(512 / Rt, 1);
  const int64_t iters = (m_max + gmax - 1) / gmax;
  int64_t G = (m_max + iters - 1) / iters;
  G = (G + quantum - 1) / quantum * quantum;
  if (G * Rt > 512) G = 512 / Rt;
  const int block = (int)std::max<int64_t>(G * Rt, 32);
  int per_sm = 0;
  cudaError_t e = grad_occupancy(scheme, block, (int)smem, &per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "gradient occupancy query");
  if (per_sm < 1) return fail(EULER_ERR_TOO_LARGE, "gradient kernel cannot be resident");
  const int64_t tiles = (R + Rt - 1) / Rt;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * h->sm_count, tiles));
  RunParams p;
  std::memset(&p, 0, sizeof p);
  p.p0 = h->d_p0;
  p.lam = h->d_lam;
  p.h = (float)dt;
  p.K = (int32_t)K;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  set_round_keys(p.rk, p.key0, p.key1);
  p.R = R;
  p.rep_begin = rep_begin;
  p.scheme = scheme;
  p.tile_reps = Rt;
  p.num_tiles = tiles;
  p.cap = h->opt[EULER_OPT_SAMPLER_CAP] > 0 ? (int32_t)h->opt[EULER_OPT_SAMPLER_CAP] : 1000;
  p.stats = stats;
  p.err = h->d_err;
  p.wait_limit = (int64_t)1 << 25;
  p.p0f = h->d_p0f;
  p.dlam = h->d_dlam;
  p.scores = scores;
  p.muh = h->d_muh;
  p.dep_mode = 0;
  p.mtab = h->mtab();
  CUDA_TRY(cudaMemsetAsync(stats, 0, sizeof(int64_t) * (size_t)euler_stats_len(h->n, R), s));
  e = launch_persistent_grad(h->tables(), p, grid, block, (int)smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "gradient kernel launch");
  e = launch_grad_reduce(h->n, R, dt, stats, scores, h->d_gpartial, grad, value, grad_var,
                                       h->opt[EULER_OPT_GRAD_CENTER] > 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

int euler_net_simulate_average(euler_net* h, double dt, double T, int64_t R, uint64_t seed,
                               int64_t rep_begin, double* stats_avg, int64_t* stats_b,
                               int64_t* stats_f, void* stream) try {
  if (!h || !stats_avg || R < 0) return fail(EULER_ERR_ARG, "bad average-scheme arguments");
  const size_t len = (size_t)euler_stats_len(h->n, R);
  if (!stats_b || !stats_f) {
    if (len > h->avg_cap || !h->d_avg_b) {
      cudaFree(h->d_avg_b);
      cudaFree(h->d_avg_f);
      h->d_avg_b = h->d_avg_f = nullptr;
      CUDA_TRY(cudaMalloc(&h->d_avg_b, sizeof(int64_t) * std::max<size_t>(len, 1)));
      CUDA_TRY(cudaMalloc(&h->d_avg_f, sizeof(int64_t) * std::max<size_t>(len, 1)));
      h->avg_cap = len;
    }
    if (!stats_b) stats_b = h->d_avg_b;
    if (!stats_f) stats_f = h->d_avg_f;
  }
  int rc = euler_net_simulate(h, EULER_BACKWARD, dt, T, R, seed, rep_begin, stats_b, stream);
  if (rc) return rc;
  rc = euler_net_simulate(h, EULER_FORWARD, dt, T, R, seed, rep_begin, stats_f, stream);
  if (rc) return rc;
  cudaError_t e = launch_average(stats_b, stats_f, stats_avg, (int64_t)len,
                                 reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "average kernel launch");
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

double euler_net_select_dt(const euler_net* h, double alpha) {
  if (!h) return -1.0;
  double mu_max = 0.0;
  int32_t m_max = 1;
  for (int32_t i = 0; i < h->n; ++i) {
    mu_max = std::max(mu_max, h->mu[i]);
    m_max = std::max(m_max, h->servers[i]);
  }
  if (!(alpha > 0.0)) alpha = 0.4 / std::sqrt((double)m_max);
  return alpha / mu_max;
}

int euler_net_status(euler_net* h, void* stream) {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaStreamSynchronize(s));
  unsigned bits = 0;
  CUDA_TRY(cudaMemcpy(&bits, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(unsigned)));
  if (bits & kErrSamplerCap) return fail(EULER_ERR_SAMPLER_CAP, "a sampler rejection loop hit its cap");
  if (bits & kErrOverflow) return fail(EULER_ERR_OVERFLOW, "a station count exceeded 2^30");
  if (bits & kErrStall) return fail(EULER_ERR_STALL, "a wait between warps of the pipelined kernel timed out");
  return EULER_OK;
}

int euler_net_simulate_host(euler_net* h, int32_t scheme, double dt, double T, int64_t R,
                            uint64_t seed, int64_t rep_begin, int64_t* stats_host, void* stream) try {
  if (!h || !stats_host) return fail(EULER_ERR_ARG, "handle or stats is NULL");
  const size_t bytes = sizeof(int64_t) * (size_t)euler_stats_len(h->n, R);
  int64_t* d_stats = nullptr;
  CUDA_TRY(cudaMalloc(&d_stats, bytes));
  int rc = euler_net_simulate(h, scheme, dt, T, R, seed, rep_begin, d_stats, stream);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (rc == EULER_OK) {
    cudaError_t e = cudaMemcpyAsync(stats_host, d_stats, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "stats copy");
  }
  const int st = euler_net_status(h, stream);
  cudaFree(d_stats);
  return rc ? rc : st;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

}  // extern "C"
