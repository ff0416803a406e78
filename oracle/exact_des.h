/*
 * exact_des.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Exact event-by-event simulation (DES) of the continuous-time Markovian
 * queueing network that the Euler schemes approximate (Sec. 2): stations
 * with m_i exponential servers of rate mu_i (FCFS, infinite waiting room),
 * Markovian routing p_ij with exit probability 1 - sum_j p_ij, external
 * Poisson arrivals of time-varying rate lambda_i(t), an optional staffing
 * schedule m_i(t).  Used to check the Euler schemes against the process they
 * approximate (the backward / forward bracketing of Sec. 2.3 and Theorem 1,
 * the error's decay in h) and as the second timed CPU baseline.
 *
 * Only the test suite and the CPU-baseline leg of the benchmark may load it.
 */
#ifndef EXACT_DES_H
#define EXACT_DES_H
#include <stdint.h>

#include "euler_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Simulate R replications (indices rep_begin ...) over (0, T] and observe the
 * state at the Euler grid t_tau = tau dt, tau = 1..K (K as eo_num_steps).
 * stats: the layout of eo_simulate, with
 *   Q_i = sum_tau N_i(t_tau), B_i = sum_tau min(N_i(t_tau), m_i(t_tau)),
 *   D_i, X_i, A_i = service completions, exits and external arrivals in (0, K dt],
 *   per replication the sums over stations, and N_i(K dt) summed over replications.
 * trace_N (optional): [K][n][R] int32 of N_i(t_tau).
 * events (optional): total events processed (arrival candidates of the
 * thinning included).  Returns EO_OK or an EO_ERR_* code. */
int eo_des_simulate(const eo_net* net, double dt, double T, int64_t R, uint64_t seed,
                    int64_t rep_begin, int64_t* stats, int32_t* trace_N, int64_t* events);

/* Sojourn time of a tagged customer that joins `station` at time t0 in each
 * replication (FCFS; exponential services, so a service completion at its
 * station is its own with probability 1 / busy servers while it is in
 * service; it follows the departing customer's routing draw).  out[r]: the
 * time from t0 to its exit, or -1 if it is still in the network at K dt.
 * Constant staffing only.  stats (optional): the run's statistics. */
int eo_des_sojourn(const eo_net* net, double dt, double T, int64_t R, uint64_t seed,
                   int64_t rep_begin, int32_t station, double t0, double* out, int64_t* stats);

#ifdef __cplusplus
}
#endif
#endif
