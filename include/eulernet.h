/*
 * eulernet.h -- C ABI of the GB300 (sm_103a) Euler-approximation simulator
 * for feedforward Markovian queueing networks.
 *
 * Method: Hong, Song & Wang, "Fast Discrete-Event Simulation of Markovian
 * Queueing Networks through Euler Approximation" (arXiv 2402.13259).
 *   - one Euler step of a network, backward scheme: Sec. 2.2 (task list 1-4),
 *     Algorithm 2;
 *   - one Euler step, forward scheme: Sec. 2.2 (task list 1-4), Algorithm 3,
 *     taken node by node in flow order for a feedforward network;
 *   - external arrivals per step: Sec. 2.1.1 (Poisson count with mean the
 *     integral of lambda_i over the step);
 *   - departures per step: GenerateDeparture, Lemma 1 / Algorithm 1;
 *   - routing: the multinomial split of Sec. 2.2.
 *
 * Conventions.
 *   - Every function returns EULER_OK (0) or a negative EULER_ERR_* code and
 *     never aborts; euler_net_last_error() returns a thread-local message for
 *     the last failure on the calling thread.
 *   - Host pointers are read during the call only and never retained.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     results are written asynchronously on the given stream (a cudaStream_t
 *     passed as void*, NULL = the legacy default stream).
 *   - Randomness: Philox4x32-10 keyed by (seed; replication, step, station,
 *     purpose).  A replication's results do not depend on the launch shape,
 *     on the tile it ran in or on which other replications ran with it.
 */
#ifndef EULERNET_H
#define EULERNET_H

#include <stdint.h>

#if defined(__GNUC__)
#define EULERNET_API __attribute__((visibility("default")))
#else
#define EULERNET_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  EULER_OK = 0,
  EULER_ERR_ARG = -1,             /* invalid argument (reported synchronously)    */
  EULER_ERR_NOT_FEEDFORWARD = -2, /* routing graph has a cycle                    */
  EULER_ERR_CUDA = -3,            /* a CUDA runtime call failed                   */
  EULER_ERR_OOM = -4,             /* device allocation failed                     */
  EULER_ERR_SAMPLER_CAP = -5,     /* a rejection loop hit its iteration cap       */
  EULER_ERR_OVERFLOW = -6,        /* a station count exceeded 2^30                */
  EULER_ERR_TOO_LARGE = -7,       /* sizes beyond this library's index ranges     */
  EULER_ERR_STALL = -8            /* a bounded wait between warps timed out       */
};

enum { EULER_BACKWARD = 0, EULER_FORWARD = 1 };
enum { EULER_ARR_NONE = 0, EULER_ARR_SINUSOID = 1, EULER_ARR_TABLE = 2 };

/* External arrival rate lambda_i(t) (Sec. 2.2, "customers arriving at the
 * i-th node from outside ... Poisson process with rate lambda_i", allowed to
 * vary in time, Sec. 2.1).
 *   EULER_ARR_SINUSOID: lambda_i(t) = w[i] * a * (1 + b sin(2 pi t / period + phase))
 *   EULER_ARR_TABLE:    piecewise linear through (j * tab_dt, table[j*n + i]),
 *                       j = 0..table_len-1, held constant after the last point.
 * The per-step mean is the exact integral of lambda_i over the step,
 * computed in double on the host. */
typedef struct {
  int32_t kind;
  const double* w;  /* [n] (sinusoid)                  */
  double a, b, period, phase;
  const double* table; /* [table_len][n] (table)       */
  int32_t table_len;
  double tab_dt;
} euler_arrivals;

typedef struct euler_net euler_net; /* opaque; owns device copies of the tables */

/* Build a network (host only, plus a one-time upload of immutable tables to
 * the current device).
 *   n        number of stations, 1 <= n < 2^24
 *   row_ptr  [n+1] CSR offsets of the routing matrix P (row i = station i)
 *   col      [nnz] destination station of each edge (no self loops)
 *   prob     [nnz] p_ij in [0,1]; exit probability p_i_exit = 1 - row sum,
 *            row sums may not exceed 1 + 1e-12
 *   servers  [n] m_i >= 1 (constant in time)
 *   mu       [n] service rate per server, finite and > 0
 *   arrivals external arrival rates (may be NULL: no external arrivals)
 *   N0       [n] initial customers per station, or NULL for an empty network
 * The graph must be feedforward (acyclic); stations are grouped into levels
 * (longest path from a source) for the forward scheme.
 * Errors: EULER_ERR_ARG, EULER_ERR_NOT_FEEDFORWARD, EULER_ERR_OOM,
 * EULER_ERR_CUDA.  On error *out is set to NULL. */
EULERNET_API int euler_net_create(euler_net** out, int32_t n, const int32_t* row_ptr, const int32_t* col,
                     const double* prob, const int32_t* servers, const double* mu,
                     const euler_arrivals* arrivals, const int32_t* N0);

/* Number of int64 entries of the stats buffer for n stations and R
 * replications: 6n + 4R. */
EULERNET_API int64_t euler_stats_len(int32_t n, int64_t replications);

/* Simulate `replications` independent replications of the backward
 * (Algorithm 2) or forward (Algorithm 3) scheme with step dt over
 * K = ceil(T/dt - 1e-9) steps, replication indices rep_begin ..
 * rep_begin + replications - 1 (the index keys the random streams, so a
 * range can be split across calls or devices and give identical results).
 *
 * stats: caller-owned DEVICE buffer of euler_stats_len(n, R) int64, fully
 * overwritten, with the sums over steps tau = 1..K of post-update values:
 *   [n][5]  per station  {Q_i = sum N, B_i = sum min(N, m_i), D_i = sum D,
 *                         X_i = sum exits, A_i = sum external arrivals}
 *   [R][4]  per replication {Q_r, D_r, X_r, A_r} (also summed over stations)
 *   [n]     N_K summed over replications.
 *
 * Asynchronous on cuda_stream.  Argument errors are returned synchronously;
 * device-side errors (EULER_ERR_SAMPLER_CAP, EULER_ERR_OVERFLOW) are latched
 * in the handle and returned by euler_net_status().  Calls on one handle must
 * not overlap on different streams (the handle's per-call tables and error
 * word are shared).  The handle caches the per-dt tables of its last call. */
EULERNET_API int euler_net_simulate(euler_net* net, int32_t scheme, double dt, double T,
                       int64_t replications, uint64_t seed, int64_t rep_begin,
                       int64_t* stats, void* cuda_stream);

/* Same as euler_net_simulate with HOST input and output: copies nothing in
 * (the network already lives on the device), allocates a temporary device
 * stats buffer, runs, copies the stats back into host memory `stats_host`
 * and synchronises.  Returns the device-side status as well. */
EULERNET_API int euler_net_simulate_host(euler_net* net, int32_t scheme, double dt, double T,
                            int64_t replications, uint64_t seed, int64_t rep_begin,
                            int64_t* stats_host, void* cuda_stream);

/* Same computation and results as euler_net_simulate, for callers that
 * cannot allocate device memory while they run (an application with a
 * device-memory budget fixed at start-up, a plug-in whose host owns the
 * allocator, a latency-critical loop where a cudaMalloc/cudaFree, which may
 * synchronise the device, is not acceptable).  The paper has no counterpart:
 * this is a deployment variant of the same step.
 *
 * It allocates nothing: its scratch (replication state, routed counts,
 * partial sums, per-step tables) lives in one 64 MiB area that the library
 * reserves on every GPU that loads it, held until the process exits.  The
 * handle must have been created beforehand (creation allocates) on the
 * current device, and `stats` is the caller's device buffer as for
 * euler_net_simulate.  The first call on a device also looks up the scratch
 * address for that device; make that first call before any stream capture.
 * Runs that need more than 64 MiB of scratch (about 4(n+E)R bytes plus 32R
 * plus 4K per external station) return EULER_ERR_TOO_LARGE.  All calls
 * share the scratch and it keeps the previous call's contents: the call
 * resets what must start at zero, and calls that overlap on the GPU (other
 * streams, other threads) race and must not be issued.  The handle's device
 * must be the current device (EULER_ERR_ARG otherwise).  The per-step tables
 * (arrival means, departure constants, staffing rows) stay in the scratch:
 * a call with the same handle, unchanged since, and the same (dt, T) as the
 * previous call on this device reuses them and is asynchronous on
 * cuda_stream; any other call stages them from host memory and synchronises
 * cuda_stream while it does.  Device-side errors are returned by
 * euler_net_status. */
EULERNET_API int euler_net_simulate_noalloc(euler_net* net, int32_t scheme, double dt, double T,
                                            int64_t replications, uint64_t seed, int64_t rep_begin,
                                            int64_t* stats, void* cuda_stream);

/* ---- Average scheme and step-size rule ---- */

/* The average scheme (Sec. 7.1: backward and forward run side by side and
 * their customer counts averaged): runs both schemes on the same random
 * streams (common random numbers) into the caller's DEVICE buffers stats_b and
 * stats_f (int64, layout of euler_net_simulate, either may be NULL to use
 * internal scratch) and writes stats_avg (DEVICE double, same layout) =
 * (stats_b + stats_f) / 2.  Asynchronous on cuda_stream. */
EULERNET_API int euler_net_simulate_average(euler_net* net, double dt, double T,
                                            int64_t replications, uint64_t seed,
                                            int64_t rep_begin, double* stats_avg,
                                            int64_t* stats_b, int64_t* stats_f, void* cuda_stream);

/* Step-size selection rule (Sec. 5.4): h = alpha / max_i mu_i.  alpha <= 0
 * takes the experiments' alpha = 0.4 / sqrt(max_i m_i) (Sec. 7.4).  Returns
 * the step, or a negative value for a NULL handle. */
EULERNET_API double euler_net_select_dt(const euler_net* net, double alpha);

/* ---- Likelihood-ratio (score-function) gradients ---- */

/* Gradients of the two performance measures, per replication
 *   L_1 = dt * sum_{tau, i} N_{tau,i}   (time-integrated total number in system)
 *   L_2 = sum_{tau, i} D_{tau,i}        (total station departures)
 * with respect to theta = (mu_1 .. mu_n, a, b, phase), the service rates and
 * the three parameters of sinusoid arrivals (zero for table arrivals).  The
 * paper has no gradients; the estimator is the likelihood-ratio one:
 * grad[m][c] = mean_r L_m(r) S_r[c], S_r = sum over the replication's draws of
 * d log p(draw)/d theta (float32 terms, float64 sums), which uses the laws of
 * the method's own draws: Poisson arrivals (Sec. 2.1.1), the binomial and
 * Erlang laws of GenerateDeparture (Lemma 1, Algorithm 1).
 *   grad      DEVICE [2][n+3] double, mean of L_m S
 *   value     DEVICE [2] double, mean of L_m
 *   grad_var  DEVICE [2][n+3] double variance of the mean, or NULL
 *   scores    DEVICE [R][n+3] double per-replication scores out, or NULL
 *   stats     DEVICE stats buffer (as euler_net_simulate) out, or NULL
 * Sums over replications run in blocks of 32 (ascending), then over blocks in
 * ascending order, so results do not depend on the launch.  Asynchronous on
 * cuda_stream; EULER_ERR_TOO_LARGE when a tile with its score sums does not
 * fit in shared memory. */
EULERNET_API int euler_net_grad(euler_net* net, int32_t scheme, double dt, double T,
                                int64_t replications, uint64_t seed, int64_t rep_begin,
                                double* grad, double* value, double* grad_var, double* scores,
                                int64_t* stats, void* cuda_stream);

/* ---- Checkpoint / resume ---- */

/* Steps step_begin+1 .. K of the run that euler_net_simulate(net, scheme, dt,
 * T, replications, seed, rep_begin) describes, started from the checkpoint
 * state_in = N_{step_begin}.  Every draw is keyed by (seed, station, step,
 * replication), so the counts N after a step are a complete checkpoint: the
 * statistics of the parts of a run split at any steps add up to those of the
 * uninterrupted run (the N_K row belongs to the last part), and the last
 * part's N_K is the same, bit for bit.  (The paper has no checkpointing.)
 *   step_begin  0 <= step_begin <= K
 *   state_in    DEVICE [n][replications] int32: N_{step_begin} of station i
 *               and replication r at i * replications + r; NULL = the
 *               network's N0 in every replication
 *   state_out   DEVICE [n][replications] int32 out: N_K; or NULL
 *   stats       DEVICE stats buffer (the layout of euler_net_simulate), the
 *               sums over steps step_begin+1 .. K only
 * Runs in the HBM-state form at any size.  Asynchronous on cuda_stream;
 * errors as euler_net_simulate, EULER_ERR_ARG for step_begin outside [0, K]. */
EULERNET_API int euler_net_simulate_resume(euler_net* net, int32_t scheme, double dt, double T,
                                           int64_t replications, uint64_t seed, int64_t rep_begin,
                                           int64_t step_begin, const int32_t* state_in,
                                           int32_t* state_out, int64_t* stats, void* cuda_stream);

/* Coupled gradient: central differences under common random numbers, with
 * checkpointed replay (an extension; the paper has no gradients).
 * theta = (mu_0 .. mu_{n-1}, s_0 .. s_{W-1}) where s_w multiplies the external
 * arrival means Lambda_tau,i of the steps of window w, tau = floor(w K / W) + 1
 * .. floor((w + 1) K / W), at s = 1.  For parameter c the run is repeated at
 * theta_c (1 + delta) and theta_c (1 - delta) with the same seed, so both use
 * the same draws and their sample paths stay coupled; per replication
 * d_m = (L_m^+ - L_m^-) / (2 delta theta_c), with L_1 = dt sum N and
 * L_2 = sum D over stations and steps (the measures of euler_net_grad).  A
 * window perturbation leaves every step before the window unchanged, so its
 * two runs replay from the base run's checkpoint at the window's first step
 * (one base pass writes the W - 1 checkpoints into [W-1][n][R] int32 of
 * device scratch).
 *   windows   W, 1 <= W <= K
 *   delta     relative perturbation, 0 < delta <= 1/2
 *   params    HOST [n_params] indices into theta, or NULL for all n + W
 *             (n_params must then be n + W)
 *   grad      DEVICE [2][n_params] double out: mean over replications of d_m
 *   grad_var  DEVICE [2][n_params] double out: variance of that mean, or NULL
 * d is summed in int64 (exact), d^2 in double in a fixed order.  Synchronous:
 * returns when grad and grad_var are written; device-side sampler errors are
 * latched as for euler_net_simulate.  EULER_ERR_ARG for replications < 1,
 * W outside [1, K], delta outside (0, 1/2] or an index out of range. */
EULERNET_API int euler_net_grad_coupled(euler_net* net, int32_t scheme, double dt, double T,
                                        int64_t replications, uint64_t seed, int64_t rep_begin,
                                        int32_t windows, double delta, const int32_t* params,
                                        int32_t n_params, double* grad, double* grad_var,
                                        void* cuda_stream);

/* ---- Sojourn times (Sec. 6, Algorithm 4) ---- */

/* Sojourn times of tagged customers that enter `station` during step tau0
 * (the interval ((tau0-1) dt, tau0 dt], 1 <= tau0 <= K), `samples` tagged
 * customers per replication, sampled on the replications' own Euler sample
 * paths (those euler_net_simulate produces with the same arguments) by
 * Algorithm 4: a customer waits at a station while more than m_i customers
 * are ahead of or at its place (its place is N_tau,i after the step it
 * arrived in), and in service it stays through a step with the probability
 * of Lemma 3 given that step's departure draw (input x, output D); leaving,
 * it follows the step's routed counts R_e / D or exits.  Each step counts h.
 *   sojourn  DEVICE [R][samples] int32 out: the sojourn in steps (> 0) if the
 *            customer left by step K, else minus the steps accounted (<= 0,
 *            censored at the horizon)
 *   stats    DEVICE stats buffer of the sample paths (as euler_net_simulate),
 *            or NULL
 * The random choices use the Philox stream (seed, purpose 3, sample index,
 * step, rep_begin + r): the first uniform decides the stay, the second word
 * picks the departing customer.  Results do not depend on the launch.
 * Asynchronous on cuda_stream.  EULER_ERR_ARG for a station or tau0 out of
 * range or samples outside [1, 65536]; EULER_ERR_TOO_LARGE when a tile with
 * its customers does not fit in shared memory. */
EULERNET_API int euler_net_sojourn(euler_net* net, int32_t scheme, double dt, double T,
                                   int64_t replications, uint64_t seed, int64_t rep_begin,
                                   int32_t station, int64_t tau0, int32_t samples, int32_t* sojourn,
                                   int64_t* stats, void* cuda_stream);

/* ---- Batched form: many independent networks in one persistent launch ---- */

/* One simulation request of a batch (see euler_net_simulate for the fields). */
typedef struct {
  int32_t scheme;
  double dt, T;
  int64_t replications;
  uint64_t seed;
  int64_t rep_begin;
} euler_run;

typedef struct euler_batch euler_batch; /* opaque */

/* Prepare `count` runs, runs[j] on network nets[j] (host planning plus
 * uploads of the per-run tables and the work queue; the handles must stay
 * alive until euler_batch_destroy).  A handle may appear several times only
 * with the same (dt, T).  A network with n x replications >= 2^18 units per
 * step (the threshold the autotuner may move) fills the GPU by itself and
 * runs in the HBM form of euler_net_simulate (per-step kernels replayed from
 * CUDA graphs), these networks one after another; the others share one
 * persistent launch whose work items are (network, tile of replications),
 * ordered by decreasing cost, with per-network tile sizes that fill the
 * block.  Errors: EULER_ERR_ARG, EULER_ERR_TOO_LARGE (a network whose
 * smallest tile does not fit in shared memory), EULER_ERR_CUDA,
 * EULER_ERR_OOM. */
EULERNET_API int euler_batch_create(euler_batch** out, euler_net* const* nets,
                                    const euler_run* runs, int32_t count);

/* Time launch shapes on shortened horizons and keep the fastest: the
 * persistent launch's threads per block (stations per CTA), shared-memory
 * budget per CTA and tile scale (replications per tile, x 1/2, 1, 2); the HBM
 * form's threads per step kernel and slots per graph replay (steps per
 * launch, 16 / 32 / 64), on up to six of its networks; then the n x
 * replications threshold between the two kinds (2^16, 2^18, 2^20 or none).
 * Synchronises `cuda_stream`; returns the persistent launch's block size in
 * *block_out (may be NULL). */
EULERNET_API int euler_batch_autotune(euler_batch* b, void* cuda_stream, int32_t* block_out);

/* Run every request: stats[j] is run j's caller-owned DEVICE buffer of
 * euler_stats_len(n_j, R_j) int64, laid out as for euler_net_simulate.  The
 * persistent part (zeroing of every stats buffer plus one persistent kernel
 * per scheme) is captured once in a CUDA graph and replayed; a call with
 * other stats pointers re-captures.  The HBM-form networks follow on the
 * same stream, each replaying its own graph of per-step kernels.  Results
 * equal one euler_net_simulate call per request.  Asynchronous on
 * cuda_stream; device-side errors via euler_batch_status. */
EULERNET_API int euler_batch_run(euler_batch* b, int64_t* const* stats, void* cuda_stream);

/* The batch's current plan (after euler_batch_create, or the autotuner's
 * choice): *hbm_networks = requests run in the HBM form, *hbm_min_units =
 * their n x replications threshold (0: none), *critical_path = 1 if the
 * critical-path rule moves long work items to the HBM form, *block and
 * *tile_shift = the persistent launch's threads per block and tile scale
 * (replications per tile x 2^tile_shift), *hbm_block and *graph_steps = the
 * HBM form's threads per step kernel and slots per graph replay.  Any output
 * pointer may be NULL.  Returns EULER_ERR_ARG for a NULL batch. */
EULERNET_API int euler_batch_info(const euler_batch* b, int32_t* hbm_networks, int64_t* hbm_min_units,
                                  int32_t* critical_path, int32_t* block, int32_t* tile_shift,
                                  int32_t* hbm_block, int32_t* graph_steps);

/* Synchronise and return the first device-side error of any run (clears them). */
EULERNET_API int euler_batch_status(euler_batch* b, void* cuda_stream);

EULERNET_API void euler_batch_destroy(euler_batch* b);

/* Convenience: create, run once, synchronise, destroy. */
EULERNET_API int euler_net_batch_simulate(euler_net* const* nets, const euler_run* runs,
                                          int32_t count, int64_t* const* stats, void* cuda_stream);

/* Synchronise `cuda_stream`, then return and clear the latched device-side
 * status of the handle's previous calls (EULER_OK if none failed). */
EULERNET_API int euler_net_status(euler_net* net, void* cuda_stream);

/* Tuning and testing options (see EULER_OPT_*); value < 0 restores the
 * default.  Returns EULER_OK or EULER_ERR_ARG. */
enum {
  EULER_OPT_FORM = 0,        /* 0 = auto (2 when n x replications >= 2^18,
                                else 1; 2 also when a tile does not fit in
                                shared memory), 1 = persistent shared-memory
                                kernel with block barriers, 2 = per-step
                                kernels over HBM state replayed from a CUDA
                                graph (forward scheme: one skewed launch per
                                step for all stations), 3 = level-pipelined
                                shared-memory kernel.  All forms give the same
                                results bit for bit.                           */
  EULER_OPT_TILE_REPS = 1,   /* replications per tile (power of two)           */
  EULER_OPT_BLOCK = 2,       /* threads per block (HBM form: default 256)      */
  EULER_OPT_GRID = 3,        /* blocks of the persistent kernel (0 = auto)     */
  EULER_OPT_SAMPLER_CAP = 4, /* rejection-loop iteration cap (default 1000)    */
  EULER_OPT_GRAPH_STEPS = 5, /* steps captured per CUDA graph (HBM form)       */
  EULER_OPT_PIPE_WARPS = 6,  /* warps per tile of the pipelined form (<= 16)   */
  EULER_OPT_WAIT_LIMIT = 7,  /* polls before an inter-warp wait of the
                                pipelined form gives up (default 2^25, about
                                2-4 s); then EULER_ERR_STALL                   */
  EULER_OPT_TEST_STALL = 8,  /* testing only: nonzero makes every warp of the
                                pipelined form withhold its progress, so the
                                warps' bounded waits run out                  */
  EULER_OPT_WAIT_SLEEP = 9,  /* nanoseconds between polls of an inter-warp
                                wait of the pipelined form (default 64)       */
  EULER_OPT_DEPARTURE = 10,  /* departure sampler: 0 = exact (Lemma 1,
                                Algorithm 1), 1 = Eq. (1) D = min(x,
                                Poisson(min(x, m) mu h)), 2 = Eq. (2)
                                (binomial for x <= m, Eq. (1) otherwise); the
                                biased modes are for speed/bias studies and
                                are not available to euler_net_grad           */
  EULER_OPT_GRAD_CENTER = 11, /* euler_net_grad's estimator: 0 = mean of L S,
                                1 = centred, mean of (L - mean L) S: the same
                                expectation (E[S] = 0), lower variance when L
                                varies little around a large mean             */
  EULER_OPT_HBM_CHUNK = 12   /* HBM form: replications run together over the
                                whole horizon before the next chunk (default:
                                as many as keep the state within ~64 MiB of
                                L2, at least 2^18 / n); results do not depend
                                on it                                          */
};
EULERNET_API int euler_net_set_option(euler_net* net, int32_t option, int64_t value);

/* Time-varying staffing (Sec. 2.1.2): m_i(t) = table[j*n + i] for
 * j = min(floor(t / tab_dt), len - 1), all entries >= 1.  A step uses the
 * servers at its start time, so staffing changes should fall on step
 * boundaries (the paper places a boundary at each change); customers whose
 * server is withdrawn simply wait again (the state is a count).  NULL or
 * len = 0 returns to the constant servers of euler_net_create.  Host copy;
 * applies to later calls. */
EULERNET_API int euler_net_set_servers_schedule(euler_net* net, const int32_t* table, int32_t len,
                                                double tab_dt);

/* Describe the launch the next euler_net_simulate would make for these
 * sizes: form (1, 2 or 3), tile replications, block, grid, shared bytes.
 * Host only; no device work. */
EULERNET_API int euler_net_plan(euler_net* net, int32_t scheme, int64_t replications, int32_t* form,
                   int32_t* tile_reps, int32_t* block, int32_t* grid, int32_t* smem_bytes);

/* Host-to-device bytes this handle has copied so far (network tables at
 * creation plus the per-(dt, T) step tables), or -1 for a NULL handle. */
EULERNET_API int64_t euler_net_h2d_bytes(const euler_net* net);

/* Number of Euler steps used for (dt, T): ceil(T/dt - 1e-9), at least 1. */
EULERNET_API int64_t euler_num_steps(double dt, double T);

EULERNET_API void euler_net_destroy(euler_net* net);
EULERNET_API const char* euler_net_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EULERNET_H */
