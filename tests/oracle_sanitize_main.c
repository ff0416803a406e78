/*
 * oracle_sanitize_main.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Drives every entry point of the CPU oracle and the exact DES on small
 * networks that reach every sampler branch (inversion and rejection
 * samplers, both branches of Algorithm 1, Eq. (1)/(2), staffing, table and
 * sinusoid arrivals, traces, scores, sojourn times, resume, the arrival
 * window), so that a build with AddressSanitizer and UndefinedBehaviorSanitizer
 * reports any out-of-bounds access, use of freed memory or undefined
 * arithmetic.  Exit status 0 and "ok" when every call returned EO_OK.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "euler_oracle.h"
#include "exact_des.h"

static int failures = 0;

static void expect(int rc, const char* what) {
  if (rc != EO_OK) {
    fprintf(stderr, "%s returned %d\n", what, rc);
    ++failures;
  }
}

int main(void) {
  /* 4 stations: 0 -> 1 (0.6), 0 -> 2 (0.3), 1 -> 3 (1.0), 2 -> 3 (0.5); few
     servers at 0 and 1 so that x > m is common, many at 3 and a large rate
     at 2 so that the rejection samplers run */
  const int32_t n = 4;
  const int32_t row_ptr[5] = {0, 2, 3, 4, 4};
  const int32_t col[4] = {1, 2, 3, 3};
  const double prob[4] = {0.6, 0.3, 1.0, 0.5};
  const int32_t servers[4] = {2, 3, 400, 60};
  const double mu[4] = {2.5, 1.7, 3.0, 1.2};
  const double w[4] = {8.0, 0.0, 900.0, 0.0};
  const int32_t N0[4] = {3, 0, 350, 10};
  const int32_t sv[8] = {2, 3, 400, 60, 3, 2, 380, 70};
  const double table[12] = {6.0, 0.0, 800.0, 0.0, 9.0, 0.0, 1000.0, 0.0, 7.0, 0.0, 900.0, 0.0};
  eo_net net = {0};
  net.n = n;
  net.row_ptr = row_ptr;
  net.col = col;
  net.prob = prob;
  net.servers = servers;
  net.mu = mu;
  net.arr_kind = EO_ARR_SINUSOID;
  net.w = w;
  net.a = 1.0;
  net.b = 0.4;
  net.period = 3.0;
  net.phase = 0.3;
  net.N0 = N0;

  const double dt = 0.05, T = 2.0;
  const int64_t R = 9, K = eo_num_steps(dt, T);
  int64_t* stats = (int64_t*)calloc((size_t)(6 * n + 4 * R), sizeof(int64_t));
  int32_t* tN = (int32_t*)calloc((size_t)(K * n * R), sizeof(int32_t));
  int32_t* tD = (int32_t*)calloc((size_t)(K * n * R), sizeof(int32_t));
  int32_t* tA = (int32_t*)calloc((size_t)(K * n * R), sizeof(int32_t));
  int32_t* Nmid = (int32_t*)calloc((size_t)(n * R), sizeof(int32_t));
  int32_t* Nend = (int32_t*)calloc((size_t)(n * R), sizeof(int32_t));
  double grad[2 * 7], value[2], var[2 * 7];
  double* scores = (double*)calloc((size_t)(R * (n + 3)), sizeof(double));
  int32_t* soj = (int32_t*)calloc((size_t)(R * 3), sizeof(int32_t));
  double des_out[9];
  int64_t events = 0;

  for (int32_t scheme = 0; scheme < 2; ++scheme) {
    for (int32_t mode = 0; mode < 3; ++mode) {
      eo_set_departure_mode(mode);
      expect(eo_simulate(&net, scheme, dt, T, R, 11, 2, stats, tN, tD, tA), "eo_simulate");
    }
    eo_set_departure_mode(0);
    expect(eo_simulate_resume(&net, scheme, dt, 0.5 * T, R, 11, 2, 0, NULL, Nmid, stats),
           "eo_simulate_resume (first part)");
    expect(eo_simulate_resume(&net, scheme, dt, T, R, 11, 2, K / 2, Nmid, Nend, stats),
           "eo_simulate_resume (second part)");
    eo_set_arrival_window(3, 9, 1.05);
    expect(eo_simulate(&net, scheme, dt, T, R, 11, 2, stats, NULL, NULL, NULL), "eo_simulate (window)");
    eo_set_arrival_window(1, 0, 1.0);
    for (int32_t c = 0; c < 2; ++c) {
      eo_set_grad_center(c);
      expect(eo_grad(&net, scheme, dt, T, R, 11, 2, scores, grad, value, var), "eo_grad");
    }
    eo_set_grad_center(0);
    expect(eo_sojourn(&net, scheme, dt, T, R, 11, 2, 0, 3, 3, soj, stats), "eo_sojourn");
  }
  /* staffing schedule and table arrivals */
  net.sv_table = sv;
  net.sv_len = 2;
  net.sv_dt = 1.0;
  net.arr_kind = EO_ARR_TABLE;
  net.table = table;
  net.table_len = 3;
  net.tab_dt = 0.7;
  for (int32_t scheme = 0; scheme < 2; ++scheme)
    expect(eo_simulate(&net, scheme, dt, T, R, 12, 0, stats, tN, tD, tA), "eo_simulate (schedule)");
  expect(eo_des_simulate(&net, dt, T, 4, 13, 0, stats, tN, &events), "eo_des_simulate");
  net.sv_table = NULL;
  net.sv_len = 0;
  expect(eo_des_sojourn(&net, dt, T, 4, 13, 0, 0, 0.4, des_out, stats), "eo_des_sojourn");

  /* samplers and primitives, small and large parameters */
  int32_t iv[64];
  float fv[64];
  double routep[3] = {0.2, 0.5, 0.1};
  int32_t routes[64 * 4];
  expect(eo_draw_poisson(3.5f, 1, 64, iv), "eo_draw_poisson (inversion)");
  expect(eo_draw_poisson(250.0f, 1, 64, iv), "eo_draw_poisson (PTRS)");
  expect(eo_draw_binomial(40, 0.1f, 1, 64, iv), "eo_draw_binomial (inversion)");
  expect(eo_draw_binomial(5000, 0.3f, 1, 64, iv), "eo_draw_binomial (BTRS)");
  expect(eo_draw_binomial(5000, 0.8f, 1, 64, iv), "eo_draw_binomial (symmetric)");
  expect(eo_draw_gamma(5, 2.0f, 1, 64, fv), "eo_draw_gamma (small)");
  expect(eo_draw_gamma(40, 2.0f, 1, 64, fv), "eo_draw_gamma (Marsaglia-Tsang)");
  expect(eo_draw_normal(1, 64, fv), "eo_draw_normal");
  expect(eo_draw_departure(30, 4, 1.5, 0.2, 1, 64, iv), "eo_draw_departure");
  expect(eo_draw_route(25, 3, routep, 1, 64, routes), "eo_draw_route");
  float xs[5] = {-3.0f, 0.0f, 1e-30f, 7.5f, 80.0f}, ys[5];
  for (int32_t fn = 0; fn < 4; ++fn) eo_map_f32(fn, xs, ys, 5);
  float us[16];
  eo_uniforms(5, 1, 2, 3, 4, 16, us);
  (void)eo_sojourn_pstay(9, 2, 4);

  free(stats);
  free(tN);
  free(tD);
  free(tA);
  free(Nmid);
  free(Nend);
  free(scores);
  free(soj);
  if (failures) return 1;
  printf("ok\n");
  return 0;
}
