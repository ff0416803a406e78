// coupled.cu -- checkpoint / resume of a run, and the coupled
// (common-random-numbers) central-difference gradient that replays the
// perturbed runs from checkpoints.
//
// Every draw is keyed by (seed, purpose, station, step, replication), so the
// state N_tau of every station and replication after step tau is a complete
// checkpoint: a run of steps tau+1 .. K from it reproduces the uninterrupted
// run bit for bit.  Two runs that differ only in a parameter use the same
// draws (common random numbers), and the inversion samplers are monotone in
// their parameters, so the two sample paths stay coupled and the difference
// of their measures is small and low-variance.  A perturbation of the
// external arrival means of the steps of one time window leaves every step
// before the window unchanged: its two runs start from the base run's
// checkpoint at the window's first step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/eulernet.h"
#include "handle.h"
#include "internal.h"

using namespace eulernet;

namespace {

int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  set_last_error((std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e)).c_str());
  return e == cudaErrorMemoryAllocation ? EULER_ERR_OOM : EULER_ERR_CUDA;
}

#define CTRY(expr)                                      \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

int check_run_args(const euler_net* h, int32_t scheme, double dt, double T, int64_t R,
                   int64_t rep_begin) {
  if (!h) return fail(EULER_ERR_ARG, "handle is NULL");
  if (scheme != EULER_BACKWARD && scheme != EULER_FORWARD) return fail(EULER_ERR_ARG, "unknown scheme");
  if (!(dt > 0.0) || !(T > 0.0) || !std::isfinite(dt) || !std::isfinite(T))
    return fail(EULER_ERR_ARG, "dt and T must be finite and > 0");
  if (R < 0 || rep_begin < 0) return fail(EULER_ERR_ARG, "replications and rep_begin must be >= 0");
  if (rep_begin + R > (int64_t)1 << 32) return fail(EULER_ERR_TOO_LARGE, "replication index beyond 2^32");
  const int64_t K = euler_num_steps(dt, T);
  if (K >= (1 << 24)) return fail(EULER_ERR_TOO_LARGE, "too many steps (T/dt >= 2^24)");
  if (h->n_ex > 0 && K * (int64_t)h->n_ex > ((int64_t)1 << 31))
    return fail(EULER_ERR_TOO_LARGE, "arrival table too large");
  return EULER_OK;
}

// Steps tau0+1 .. tau_end of the scheme in the HBM form, from state_in
// (N_tau0, [n][R], or the network's N0) to state_out (N_tau_end, or
// nullptr); statistics of those steps into the caller's device buffer.
int run_range(euler_net* h, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
              int64_t rep_begin, int64_t tau0, int64_t tau_end, const int32_t* state_in,
              int32_t* state_out, int64_t* stats, cudaStream_t s) {
  CTRY(cudaMemsetAsync(stats, 0, sizeof(int64_t) * (size_t)euler_stats_len(h->n, R), s));
  if (R == 0) return EULER_OK;
  int rc = prepare_step_tables(h, dt, T, s);
  if (rc) return rc;
  RunParams p;
  std::memset(static_cast<void*>(&p), 0, sizeof p);
  p.p0 = h->d_p0;
  p.lam = h->d_lam;
  p.h = (float)dt;
  p.K = (int32_t)tau_end;
  p.tau0 = (int32_t)tau0;
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
  p.muh = h->d_muh;
  p.dep_mode = h->dep_mode();
  p.mtab = h->mtab();
  const int block = h->opt[EULER_OPT_BLOCK] > 0 ? (int)h->opt[EULER_OPT_BLOCK] : kHbmBlock;
  if (block % 32 || block > 256) return fail(EULER_ERR_ARG, "HBM-form block must be a multiple of 32 <= 256");
  HbmExtra x;
  x.state_in = state_in;
  x.state_out = state_out;
  return run_hbm_form(h, h->tables(), p, block, s, x);
}

// Per-replication differences d = L(theta + delta_c) - L(theta - delta_c)
// of the two measures (Q_r = sum N, D_r = sum D) of two runs: sum of d in
// int64 (exact), sum of d^2 in double over a fixed order (thread t takes
// replications t, t + 1024, ... ascending, then a fixed tree), then
//   grad = (S1 / R) * scale,  var = ((S2 - S1 (S1 / R)) / (R - 1)) scale^2 / R,
// scale = (dt for Q, 1 for D) / (2 delta theta_c).  One block of 1024.
__global__ void __launch_bounds__(1024) coupled_reduce_kernel(const int64_t* plus, const int64_t* minus,
                                                             int32_t n, int64_t R, double dt, double den,
                                                             int32_t k, int32_t P, double* grad,
                                                             double* var) {
  __shared__ long long s1[2][1024];
  __shared__ double s2[2][1024];
  const int t = threadIdx.x;
  long long a1[2] = {0, 0};
  double a2[2] = {0.0, 0.0};
  const int64_t* pr = plus + 5 * (int64_t)n;
  const int64_t* mr = minus + 5 * (int64_t)n;
  for (int64_t r = t; r < R; r += 1024) {
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const long long d = (long long)(pr[4 * r + m] - mr[4 * r + m]);
      a1[m] += d;
      a2[m] += (double)d * (double)d;
    }
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    s1[m][t] = a1[m];
    s2[m][t] = a2[m];
  }
  __syncthreads();
  for (int off = 512; off > 0; off >>= 1) {
    if (t < off) {
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        s1[m][t] += s1[m][t + off];
        s2[m][t] += s2[m][t + off];
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    for (int m = 0; m < 2; ++m) {
      const double S1 = (double)s1[m][0], S2 = s2[m][0];
      const double scale = (m == 0 ? dt : 1.0) / den;
      grad[m * P + k] = (S1 / (double)R) * scale;
      if (var)
        var[m * P + k] = R > 1 ? ((S2 - S1 * (S1 / (double)R)) / (double)(R - 1)) * (scale * scale) / (double)R
                               : 0.0;
    }
  }
}

// Window w of W over steps 1..K: steps lo .. hi.
void window_steps(int64_t K, int32_t W, int32_t w, int64_t* lo, int64_t* hi) {
  *lo = (int64_t)w * K / W + 1;
  *hi = (int64_t)(w + 1) * K / W;
}

// Changes one parameter of the handle in place for the perturbed runs and
// puts it back when it goes out of scope (also on an error return).
struct Perturb {
  euler_net* h;
  cudaStream_t s;
  int32_t mu_i = -1;
  double mu_old = 0.0;
  bool window = false;

  Perturb(euler_net* h_, cudaStream_t s_) : h(h_), s(s_) {}
  int set_mu(int32_t i, double v) {
    // the runs on s read the device copy: let them finish first
    CTRY(cudaStreamSynchronize(s));
    if (mu_i < 0) {
      mu_i = i;
      mu_old = h->mu[i];
    }
    h->mu[i] = v;
    const float f = (float)v;
    CTRY(cudaMemcpy(h->d_mu + i, &f, sizeof f, cudaMemcpyHostToDevice));
    h->invalidate_step_tables();  // the p0 constants and mu h depend on mu
    return EULER_OK;
  }
  void set_window(int64_t lo, int64_t hi, double factor) {
    window = true;
    h->win_lo = lo;
    h->win_hi = hi;
    h->win_factor = factor;
    h->invalidate_step_tables();
  }
  ~Perturb() {
    if (mu_i >= 0) {
      cudaStreamSynchronize(s);
      h->mu[mu_i] = mu_old;
      const float f = (float)mu_old;
      cudaMemcpy(h->d_mu + mu_i, &f, sizeof f, cudaMemcpyHostToDevice);
      h->invalidate_step_tables();
    }
    if (window) {
      h->win_lo = 1;
      h->win_hi = 0;
      h->win_factor = 1.0;
      h->invalidate_step_tables();
    }
  }
};

struct DeviceBuffer {
  void* p = nullptr;
  ~DeviceBuffer() { cudaFree(p); }
};

}  // namespace

extern "C" int euler_net_simulate_resume(euler_net* h, int32_t scheme, double dt, double T, int64_t R,
                                         uint64_t seed, int64_t rep_begin, int64_t step_begin,
                                         const int32_t* state_in, int32_t* state_out, int64_t* stats,
                                         void* stream) try {
  int rc = check_run_args(h, scheme, dt, T, R, rep_begin);
  if (rc) return rc;
  const int64_t K = euler_num_steps(dt, T);
  if (step_begin < 0 || step_begin > K) return fail(EULER_ERR_ARG, "step_begin must be in [0, K]");
  if (!stats) return fail(EULER_ERR_ARG, "stats is NULL");
  return run_range(h, scheme, dt, T, R, seed, rep_begin, step_begin, K, state_in, state_out, stats,
                   reinterpret_cast<cudaStream_t>(stream));
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}

extern "C" int euler_net_grad_coupled(euler_net* h, int32_t scheme, double dt, double T, int64_t R,
                                      uint64_t seed, int64_t rep_begin, int32_t windows, double delta,
                                      const int32_t* params, int32_t n_params, double* grad,
                                      double* grad_var, void* stream) try {
  int rc = check_run_args(h, scheme, dt, T, R, rep_begin);
  if (rc) return rc;
  const int64_t K = euler_num_steps(dt, T);
  if (R < 1) return fail(EULER_ERR_ARG, "replications must be >= 1");
  if (windows < 1 || windows > K) return fail(EULER_ERR_ARG, "windows must be in [1, K]");
  if (!(delta > 0.0) || !(delta <= 0.5)) return fail(EULER_ERR_ARG, "delta must be in (0, 1/2]");
  if (!grad) return fail(EULER_ERR_ARG, "grad is NULL");
  const int32_t P_all = h->n + windows;
  if (!params && n_params != P_all) return fail(EULER_ERR_ARG, "without params, n_params must be n + windows");
  if (n_params < 1) return fail(EULER_ERR_ARG, "n_params must be >= 1");
  std::vector<int32_t> par(n_params);
  bool any_window = false;
  for (int32_t k = 0; k < n_params; ++k) {
    par[k] = params ? params[k] : k;
    if (par[k] < 0 || par[k] >= P_all) return fail(EULER_ERR_ARG, "parameter index out of range");
    any_window = any_window || par[k] >= h->n;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t slen = (size_t)euler_stats_len(h->n, R);
  const size_t cell = (size_t)h->n * (size_t)R;
  DeviceBuffer plus, minus, ckpt;
  CTRY(cudaMalloc(&plus.p, sizeof(int64_t) * slen));
  CTRY(cudaMalloc(&minus.p, sizeof(int64_t) * slen));
  int64_t* sp = static_cast<int64_t*>(plus.p);
  int64_t* sm = static_cast<int64_t*>(minus.p);
  // checkpoints N at the start of windows 1 .. W-1 (window 0 starts from N0)
  int32_t* cp = nullptr;
  if (any_window && windows > 1) {
    CTRY(cudaMalloc(&ckpt.p, sizeof(int32_t) * cell * (size_t)(windows - 1)));
    cp = static_cast<int32_t*>(ckpt.p);
    for (int32_t w = 0; w + 1 < windows; ++w) {
      int64_t lo, hi;
      window_steps(K, windows, w, &lo, &hi);
      rc = run_range(h, scheme, dt, T, R, seed, rep_begin, lo - 1, hi, w ? cp + cell * (w - 1) : nullptr,
                     cp + cell * w, sp, s);
      if (rc) return rc;
    }
  }
  for (int32_t k = 0; k < n_params; ++k) {
    const int32_t c = par[k];
    double theta = 1.0;
    {
      Perturb pt(h, s);
      int64_t tau0 = 0;
      const int32_t* from = nullptr;
      if (c < h->n) {
        theta = h->mu[c];
        rc = pt.set_mu(c, theta * (1.0 + delta));
        if (!rc) rc = run_range(h, scheme, dt, T, R, seed, rep_begin, 0, K, nullptr, nullptr, sp, s);
        if (!rc) rc = pt.set_mu(c, theta * (1.0 - delta));
        if (!rc) rc = run_range(h, scheme, dt, T, R, seed, rep_begin, 0, K, nullptr, nullptr, sm, s);
      } else {
        const int32_t w = c - h->n;
        int64_t lo, hi;
        window_steps(K, windows, w, &lo, &hi);
        tau0 = lo - 1;
        from = w ? cp + cell * (w - 1) : nullptr;
        pt.set_window(lo, hi, 1.0 + delta);
        rc = run_range(h, scheme, dt, T, R, seed, rep_begin, tau0, K, from, nullptr, sp, s);
        if (!rc) {
          pt.set_window(lo, hi, 1.0 - delta);
          rc = run_range(h, scheme, dt, T, R, seed, rep_begin, tau0, K, from, nullptr, sm, s);
        }
      }
      if (rc) return rc;
    }
    coupled_reduce_kernel<<<1, 1024, 0, s>>>(sp, sm, h->n, R, dt, 2.0 * delta * theta, k, n_params, grad,
                                             grad_var);
    CTRY(cudaGetLastError());
  }
  CTRY(cudaStreamSynchronize(s));
  return EULER_OK;
} catch (const std::bad_alloc&) {
  return fail(EULER_ERR_OOM, "host memory allocation failed");
} catch (...) {
  return fail(EULER_ERR_CUDA, "unexpected error");
}
