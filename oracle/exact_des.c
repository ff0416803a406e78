/*
 * exact_des.c -- TEST INFRASTRUCTURE ONLY (see exact_des.h).
 *
 * The network is a continuous-time Markov chain on the station counts N:
 *   external arrival at i:    rate lambda_i(t)                 N_i += 1
 *   service completion at i:  rate min(N_i, m_i(t)) mu_i       N_i -= 1, then the
 *                             customer joins j with probability p_ij or leaves
 * (exponential services make the FCFS order irrelevant to the counts).  The
 * chain is simulated event by event: with the total rate S of the service
 * completions and a bound Lmax >= sum_i lambda_i(t), the next candidate event
 * comes after an Exp(Lmax + S) time; it is a service completion with
 * probability S / (Lmax + S), otherwise an arrival candidate at station i
 * (probability lambda_max_i / Lmax), accepted with probability
 * lambda_i(t) / lambda_max_i (thinning of a non-homogeneous Poisson process,
 * Lewis and Shedler 1979).  A staffing schedule changes m at known times; the
 * simulation stops at each change and redraws (memorylessness).
 *
 * Random numbers: Philox4x32-10 with counter (4<<24 | block, overflow count,
 * 0, replication) and key (seed lo, seed hi); 53-bit uniforms from two words.
 * Double precision throughout; libm is fine here (nothing is compared bit for
 * bit with this simulation).
 */
#include "exact_des.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint32_t key[2];
  uint32_t rep;
  uint32_t hi;   /* counts overflows of the 24-bit block index */
  uint32_t blk;
  uint32_t buf[4];
  int used;
} des_rng;

static void rng_init(des_rng* g, uint64_t seed, uint32_t rep) {
  g->key[0] = (uint32_t)seed;
  g->key[1] = (uint32_t)(seed >> 32);
  g->rep = rep;
  g->hi = 0;
  g->blk = 0;
  g->used = 4;
}

static uint32_t rng_word(des_rng* g) {
  if (g->used == 4) {
    const uint32_t c[4] = {(4u << 24) | g->blk, g->hi, 0u, g->rep};
    eo_philox4x32_10(c, g->key, g->buf);
    if (++g->blk == (1u << 24)) {
      g->blk = 0;
      g->hi++;
    }
    g->used = 0;
  }
  return g->buf[g->used++];
}

/* uniform on (0, 1): (k + 1/2) 2^-53 for a 53-bit integer k */
static double rng_u01(des_rng* g) {
  const uint64_t a = rng_word(g) >> 5, b = rng_word(g) >> 6;
  return ((double)(a * 67108864u + b) + 0.5) * (1.0 / 9007199254740992.0);
}

/* lambda_i(t) of the network's arrival description, clamped at zero */
static double rate_at(const eo_net* net, int32_t i, double t) {
  if (net->arr_kind == EO_ARR_SINUSOID) {
    const double om = 6.283185307179586 / net->period;
    const double v = net->w[i] * net->a * (1.0 + net->b * sin(om * t + net->phase));
    return v > 0.0 ? v : 0.0;
  }
  if (net->arr_kind == EO_ARR_TABLE) {
    const int32_t J = net->table_len, n = net->n;
    const double x = t / net->tab_dt;
    int64_t j = (int64_t)floor(x);
    if (j >= J - 1) return net->table[(int64_t)(J - 1) * n + i];
    if (j < 0) j = 0;
    const double y0 = net->table[j * n + i], y1 = net->table[(j + 1) * n + i];
    const double v = y0 + (y1 - y0) * (x - (double)j);
    return v > 0.0 ? v : 0.0;
  }
  return 0.0;
}

/* an upper bound of lambda_i over all t */
static double rate_bound(const eo_net* net, int32_t i) {
  if (net->arr_kind == EO_ARR_SINUSOID) {
    const double v = net->w[i] * net->a * (1.0 + fabs(net->b));
    return v > 0.0 ? v : 0.0;
  }
  if (net->arr_kind == EO_ARR_TABLE) {
    double v = 0.0;
    for (int32_t j = 0; j < net->table_len; ++j) {
      const double y = net->table[(int64_t)j * net->n + i];
      if (y > v) v = y;
    }
    return v;
  }
  return 0.0;
}

static const int32_t* servers_at_time(const eo_net* net, double t) {
  if (!net->sv_table) return net->servers;
  int64_t j = (int64_t)floor(t / net->sv_dt);
  if (j > net->sv_len - 1) j = net->sv_len - 1;
  if (j < 0) j = 0;
  return net->sv_table + j * net->n;
}

/* The simulation; with tag_station >= 0 one tagged customer joins that
 * station at time tag_t0 in every replication and its sojourn is written to
 * tag_out[r] (-1 if it is still in the network at K dt). */
static int des_run(const eo_net* net, double dt, double T, int64_t R, uint64_t seed,
                   int64_t rep_begin, int64_t* stats, int32_t* trace_N, int64_t* events,
                   int32_t tag_station, double tag_t0, double* tag_out) {
  if (!net || net->n < 1 || !net->row_ptr || !net->servers || !net->mu || !stats) return EO_ERR_ARG;
  if (!(dt > 0.0) || !(T > 0.0) || R < 0 || rep_begin < 0) return EO_ERR_ARG;
  const int32_t n = net->n;
  for (int32_t i = 0; i < n; ++i) {
    if (net->servers[i] < 1 || !(net->mu[i] > 0.0)) return EO_ERR_ARG;
    double s = 0.0;
    for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) {
      if (net->col[e] < 0 || net->col[e] >= n || !(net->prob[e] >= 0.0)) return EO_ERR_ARG;
      s += net->prob[e];
    }
    if (s > 1.0 + 1e-12) return EO_ERR_ARG;
  }
  const int64_t K = eo_num_steps(dt, T);
  const double t_end = (double)K * dt;

  int64_t* st_station = stats;
  int64_t* st_rep = stats + 5 * (int64_t)n;
  int64_t* st_NK = st_rep + 4 * R;
  memset(stats, 0, (size_t)(6 * (int64_t)n + 4 * R) * sizeof(int64_t));

  double* lmax = (double*)malloc((size_t)n * sizeof(double));
  double* srate = (double*)malloc((size_t)n * sizeof(double));
  int64_t* N = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  double Lmax = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    lmax[i] = rate_bound(net, i);
    Lmax += lmax[i];
  }
  int64_t nev = 0;

  for (int64_t r = 0; r < R; ++r) {
    des_rng g;
    rng_init(&g, seed, (uint32_t)(rep_begin + r));
    for (int32_t i = 0; i < n; ++i) N[i] = net->N0 ? net->N0[i] : 0;
    double t = 0.0;
    int64_t tau = 1;  /* next observation index */
    double next_change = net->sv_table ? net->sv_dt : INFINITY;
    const int32_t* m = servers_at_time(net, 0.0);
    int64_t* sr = st_rep + 4 * r;
    /* tagged customer: station (-1 before it joins / after it leaves) and its
       place (customers ahead of it plus one; <= m: in service) */
    int32_t tag_at = -1;
    int64_t tag_pos = 0;
    int tag_pending = tag_station >= 0;
    if (tag_out) tag_out[r] = -1.0;
    for (;;) {
      double S = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        const int64_t busy = N[i] < m[i] ? N[i] : m[i];
        srate[i] = (double)busy * net->mu[i];
        S += srate[i];
      }
      const double Rtot = Lmax + S;
      double t_next = Rtot > 0.0 ? t - log(rng_u01(&g)) / Rtot : INFINITY;
      int change = next_change < t_next && next_change <= t_end;
      double t_stop = change ? next_change : t_next;
      const int join = tag_pending && tag_t0 < t_stop && tag_t0 <= t_end;
      if (join) {  /* the tagged customer joins before the next event: redraw after */
        change = 0;
        t_stop = tag_t0;
      }
      /* observations in (t, t_stop] see the current state */
      while (tau <= K && (double)tau * dt <= t_stop) {
        const int32_t* mo = servers_at_time(net, (double)tau * dt);
        for (int32_t i = 0; i < n; ++i) {
          int64_t* ss = st_station + 5 * (int64_t)i;
          ss[0] += N[i];
          ss[1] += N[i] < mo[i] ? N[i] : mo[i];
          sr[0] += N[i];
          if (trace_N) trace_N[((tau - 1) * n + i) * R + r] = (int32_t)N[i];
        }
        ++tau;
      }
      if (t_stop > t_end) break;
      if (join) {
        t = tag_t0;
        tag_pending = 0;
        tag_at = tag_station;
        N[tag_at] += 1;
        tag_pos = N[tag_at];
        continue;
      }
      if (change) {  /* staffing changes before the next event: redraw from there */
        t = next_change;
        next_change += net->sv_dt;
        if (next_change >= (double)net->sv_len * net->sv_dt) next_change = INFINITY;
        m = servers_at_time(net, t);
        continue;
      }
      t = t_next;
      ++nev;
      double u = rng_u01(&g) * Rtot;
      if (u < Lmax) {  /* arrival candidate */
        int32_t i = 0;
        while (i < n - 1 && u >= lmax[i]) {
          u -= lmax[i];
          ++i;
        }
        if (lmax[i] > 0.0 && rng_u01(&g) * lmax[i] < rate_at(net, i, t)) {
          N[i] += 1;
          st_station[5 * (int64_t)i + 4] += 1;
          sr[3] += 1;
        }
      } else {  /* service completion */
        u -= Lmax;
        int32_t i = 0;
        while (i < n - 1 && (srate[i] <= 0.0 || u >= srate[i])) {
          u -= srate[i];
          ++i;
        }
        if (N[i] <= 0) {  /* rounding at the end of the scan: take the last busy station */
          for (i = n - 1; i > 0 && srate[i] <= 0.0; --i) {
          }
        }
        /* the tagged customer at this station: waiting, it moves up one place;
           in service, the completion is its own with probability 1 / busy */
        int tag_leaves = 0;
        if (tag_at == i) {
          const int64_t busy = N[i] < m[i] ? N[i] : m[i];
          if (tag_pos > m[i]) {
            tag_pos -= 1;
          } else if (rng_u01(&g) * (double)busy < 1.0) {
            tag_leaves = 1;
          }
        }
        N[i] -= 1;
        st_station[5 * (int64_t)i + 2] += 1;
        sr[1] += 1;
        double v = rng_u01(&g);
        int32_t dest = -1;
        for (int32_t e = net->row_ptr[i]; e < net->row_ptr[i + 1]; ++e) {
          if (v < net->prob[e]) {
            dest = net->col[e];
            break;
          }
          v -= net->prob[e];
        }
        if (dest >= 0) {
          N[dest] += 1;
        } else {
          st_station[5 * (int64_t)i + 3] += 1;
          sr[2] += 1;
        }
        if (tag_leaves) {
          if (dest >= 0) {
            tag_at = dest;
            tag_pos = N[dest];
          } else {
            tag_at = -1;
            if (tag_out) tag_out[r] = t - tag_t0;
          }
        }
      }
    }
    for (int32_t i = 0; i < n; ++i) st_NK[i] += N[i];
  }
  if (events) *events = nev;
  free(lmax);
  free(srate);
  free(N);
  return EO_OK;
}

int eo_des_simulate(const eo_net* net, double dt, double T, int64_t R, uint64_t seed,
                    int64_t rep_begin, int64_t* stats, int32_t* trace_N, int64_t* events) {
  return des_run(net, dt, T, R, seed, rep_begin, stats, trace_N, events, -1, 0.0, NULL);
}

int eo_des_sojourn(const eo_net* net, double dt, double T, int64_t R, uint64_t seed,
                   int64_t rep_begin, int32_t station, double t0, double* out, int64_t* stats) {
  if (!net || station < 0 || station >= net->n || !(t0 >= 0.0) || !out) return EO_ERR_ARG;
  if (net->sv_table) return EO_ERR_ARG;  /* constant staffing only */
  int64_t* st = stats ? stats : (int64_t*)malloc((size_t)(6 * (int64_t)net->n + 4 * R) * sizeof(int64_t));
  const int rc = des_run(net, dt, T, R, seed, rep_begin, st, NULL, NULL, station, t0, out);
  if (!stats) free(st);
  return rc;
}
