/*
 * euler_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded CPU oracle for the backward and forward Euler
 * schemes of Hong, Song & Wang, "Fast Discrete-Event Simulation of Markovian
 * Queueing Networks through Euler Approximation" (arXiv 2402.13259).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path:
 * Philox, the float math functions, the samplers and the time loop are all
 * written out again here from their published definitions.
 *
 * Passages followed (section / algorithm / equation of the paper):
 *   - external arrivals: Sec. 2.1.1 (aggregated Poisson counts over a step)
 *   - pure-departure sampler: Lemma 1 and Algorithm 1 (Sec. 4.1.3)
 *   - routing: Sec. 2.2 (multinomial split of a node's departures)
 *   - backward scheme: Sec. 2.2 task list 1-4 and Algorithm 2
 *   - forward scheme: Sec. 2.2 task list 1-4 and Algorithm 3 (node-by-node in
 *     flow order for a feedforward network)
 *   - sojourn times: Sec. 6, Algorithm 4 and Lemma 3
 *
 * The paper does not specify the random-variate generators; the sampler
 * definitions below (Philox4x32-10 keying, uniform mapping, inversion /
 * PTRS / BTRS / Marsaglia-Tsang, float32 working precision) are this
 * project's reading, and the CUDA path implements the same definitions
 * independently so that integer trajectories agree bit for bit.
 */
#ifndef EULER_ORACLE_H
#define EULER_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  EO_OK = 0,
  EO_ERR_ARG = -1,
  EO_ERR_NOT_FEEDFORWARD = -2,
  EO_ERR_SAMPLER_CAP = -5,
  EO_ERR_OVERFLOW = -6
};
enum { EO_BACKWARD = 0, EO_FORWARD = 1 };
enum { EO_ARR_NONE = 0, EO_ARR_SINUSOID = 1, EO_ARR_TABLE = 2 };

/* Network description.  All arrays are read only; nothing is retained. */
typedef struct {
  int32_t n;               /* number of stations                          */
  const int32_t* row_ptr;  /* [n+1] CSR of the routing matrix P            */
  const int32_t* col;      /* [nnz] destination station of each edge       */
  const double* prob;      /* [nnz] p_ij; exit probability = 1 - row sum   */
  const int32_t* servers;  /* [n] m_i >= 1                                 */
  const double* mu;        /* [n] mu_i > 0                                 */
  int32_t arr_kind;        /* EO_ARR_*                                     */
  /* sinusoid: lambda_i(t) = w_i * a * (1 + b*sin(2*pi*t/period + phase))  */
  const double* w;         /* [n]                                          */
  double a, b, period, phase;
  /* table: lambda_i(j*tab_dt) = table[j*n + i], piecewise linear, held
     constant after the last point                                         */
  const double* table;
  int32_t table_len;
  double tab_dt;
  const int32_t* N0;       /* [n] initial state, or NULL for an empty net  */
  /* optional staffing schedule (Sec. 2.1.2): m_i(t) = sv_table[j*n + i] for
     j = min(floor(t / sv_dt), sv_len - 1); a step uses m at its start time */
  const int32_t* sv_table;
  int32_t sv_len;
  double sv_dt;
} eo_net;

/* Departure sampler: 0 = exact (Lemma 1, Algorithm 1), 1 = Eq. (1)
 * D = min(x, Poisson(min(x, m) mu h)), 2 = Eq. (2) (binomial for x <= m,
 * Eq. (1) otherwise).  Returns the previous mode. */
int32_t eo_set_departure_mode(int32_t mode);

/* Stats layout (int64), all sums over steps tau = 1..K of post-update values:
 *   [n][5]  per station  {Q_i = sum N, B_i = sum min(N, m_i), D_i = sum D,
 *                         X_i = sum exits, A_i = sum external arrivals}
 *   [R][4]  per replication {Q_r, D_r, X_r, A_r} (sums over stations too)
 *   [n]     N_K summed over replications
 * Total 6n + 4R entries.  Trace arrays (optional, NULL to skip) are
 * [K][n][R] int32 of N (post update), D and A^ex. */
int eo_simulate(const eo_net* net, int32_t scheme, double dt, double T,
                int64_t R, uint64_t seed, int64_t rep_begin, int64_t* stats,
                int32_t* trace_N, int32_t* trace_D, int32_t* trace_A);

/* Checkpoint / resume: steps tau0+1..K from N_in = N_tau0 ([n][R],
 * replication fastest; NULL = N0), statistics over those steps only (the
 * layout of eo_simulate), N_K into N_out ([n][R] or NULL). */
int eo_simulate_resume(const eo_net* net, int32_t scheme, double dt, double T, int64_t R,
                       uint64_t seed, int64_t rep_begin, int64_t tau0, const int32_t* N_in,
                       int32_t* N_out, int64_t* stats);

/* Multiply the external arrival means Lambda_tau,i of steps lo..hi by
 * `factor` (in double, before the rounding to float) in later runs;
 * (1, 0, 1.0) switches it off. */
void eo_set_arrival_window(int64_t lo, int64_t hi, double factor);

/* Likelihood-ratio gradient of L1 = dt sum N and L2 = sum D with respect to
 * (mu_1..mu_n, a, b, phase) of the sinusoid arrivals (centred with
 * eo_set_grad_center(1)); see euler_oracle.c.
 * grad, grad_var: [2][n+3]; value: [2]; scores_out: [R][n+3] or NULL. */
int eo_grad(const eo_net* net, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
            int64_t rep_begin, double* scores_out, double* grad, double* value, double* grad_var);

/* Sojourn time of tagged customers (Sec. 6, Algorithm 4): a customer that
 * enters `station` during step tau0 (1 <= tau0 <= K), `samples` tagged
 * customers per replication, on the sample paths of eo_simulate with the same
 * arguments.  out: [R][samples] int32, the sojourn in steps if the customer
 * left by step K, else minus the steps accounted (censored, <= 0).  stats
 * (optional, 6n + 4R) receives the paths' statistics.  See euler_oracle.c. */
int eo_sojourn(const eo_net* net, int32_t scheme, double dt, double T, int64_t R, uint64_t seed,
               int64_t rep_begin, int32_t station, int64_t tau0, int32_t samples, int32_t* out,
               int64_t* stats);
/* Lemma 3: P(the tagged customer's service continues through a step | the
 * step's departure draw had input x and output d, m servers). */
float eo_sojourn_pstay(int32_t x, int32_t d, int32_t m);

/* eo_grad's estimator: 0 = mean of L S (default), 1 = centred, mean of
 * (L - mean L) S (the same expectation, as E[S] = 0; lower variance).
 * Returns the previous setting. */
int32_t eo_set_grad_center(int32_t on);

/* Number of Euler steps for a horizon: K = ceil(T/dt - 1e-9). */
int64_t eo_num_steps(double dt, double T);

/* Rejection-loop cap (default 1000); a test may lower it to exercise the
 * error path.  Returns the previous value. */
int32_t eo_set_cap(int32_t cap);

/* ---- primitives exposed for the pinning tests ---- */
void eo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float eo_expf(float x);
float eo_logf(float x);
float eo_expm1f(float x);
float eo_log1pf(float x);
void eo_map_f32(int32_t fn, const float* x, float* y, int64_t count);

/* Draw `count` variates; variate j uses the service stream keyed by (seed,
 * purpose 1, station 0, step 0, replication j) (a departure's Erlang time the
 * purpose-2 stream of the same counter).  Returns EO_OK or an error. */
int eo_draw_poisson(float lam, uint64_t seed, int64_t count, int32_t* out);
int eo_draw_binomial(int32_t n, float p, uint64_t seed, int64_t count, int32_t* out);
int eo_draw_gamma(int32_t k, float rate, uint64_t seed, int64_t count, float* out);
int eo_draw_normal(uint64_t seed, int64_t count, float* out);
int eo_draw_departure(int32_t x, int32_t m, double mu, double h, uint64_t seed,
                      int64_t count, int32_t* out);
int eo_draw_route(int32_t D, int32_t deg, const double* prob, uint64_t seed,
                  int64_t count, int32_t* out /* [count][deg+1] */);
/* First `count` uniforms of one stream (purpose, station, step, rep). */
void eo_uniforms(uint64_t seed, uint32_t purpose, uint32_t station, uint32_t step,
                 uint32_t rep, int64_t count, float* out);

/* Work counters for the algorithmic-operation model (see eo_counters_get). */
enum {
  EOC_UNITS = 0, EOC_PHILOX_BLOCKS, EOC_UNIFORMS,
  EOC_POIS_INV, EOC_POIS_INV_ITERS, EOC_POIS_PTRS, EOC_POIS_PTRS_ITERS, EOC_POIS_PTRS_LOGTESTS,
  EOC_BIN_INV, EOC_BIN_INV_ITERS, EOC_BIN_BTRS, EOC_BIN_BTRS_ITERS, EOC_BIN_BTRS_LOGTESTS,
  EOC_GAMMA_SMALL, EOC_GAMMA_SMALL_LOGS, EOC_GAMMA_MT, EOC_GAMMA_MT_ITERS, EOC_NORMAL_ITERS,
  EOC_DEP_LE_M, EOC_DEP_T_GT_H, EOC_DEP_T_LE_H, EOC_ROUTE_BINOMIALS, EOC_GATHER_EDGES,
  EOC_COUNT
};
void eo_counters_reset(void);
void eo_counters_get(int64_t out[EOC_COUNT]);

#ifdef __cplusplus
}
#endif
#endif
