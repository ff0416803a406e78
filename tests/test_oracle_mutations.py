"""The pins of test_oracle_pins.py must reject plausible slips in the oracle.

Each case plants one mistake in a copy of oracle/euler_oracle.c (checked by
test_oracle_pins.py) or oracle/exact_des.c (checked by test_oracle_des.py),
builds the copy to a temporary library and runs that suite against it in a
subprocess; the suite must fail.  Nothing here touches a GPU.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    # Algorithm 1, T > h branch: Binomial(x - m - 1, h/T) -> Binomial(x - m, h/T)
    ("alg1_tail_count", "return sample_binomial(x - m - 1, h / T, st, err);",
     "return sample_binomial(x - m, h / T, st, err);"),
    # Algorithm 1, T <= h branch: the x - m already served are dropped
    ("alg1_served_dropped", "return (x - m) + k2;", "return k2;"),
    # Lemma 1: Erlang rate m*mu written as mu
    ("erlang_rate", "float rate = (float)m * mu;", "float rate = mu;"),
    # Lemma 1(1): the x <= m test off by one.  (x < m would be no mistake: at
    # x = m the Erlang branch has T = 0 and reduces to the same binomial law.)
    ("branch_off_by_one", "if (x <= m) {\n    CNT(EOC_DEP_LE_M);", "if (x <= m + 1) {\n    CNT(EOC_DEP_LE_M);"),
    # routing: unconditional p_e used in the sequential binomials
    ("route_unconditional", "double q = suffix > 0.0 ? net->prob[e] / suffix : 0.0;",
     "double q = net->prob[e];"),
    # backward scheme: departures drawn after adding the step's arrivals
    ("backward_order", "D[i] = departure(N[i], m_t[i], mu_f[i], h_f, p0[i], muh[i], &svc, &err, &smu);",
     "D[i] = departure(N[i] + (int32_t)(lam_t[i] > 0.0f ? 1 : 0), m_t[i], mu_f[i], h_f, p0[i], muh[i], &svc, &err, &smu);"),
    # likelihood-ratio score of the x <= m binomial: dp0/dmu factor dropped
    ("score_binomial", "if (score_mu) *score_mu = h * ((k > 0 ? (float)k / p0 : 0.0f) - (float)x);",
     "if (score_mu) *score_mu = ((k > 0 ? (float)k / p0 : 0.0f) - (float)x);"),
    # likelihood-ratio score of the Erlang density: sign slip
    ("score_erlang", "float te = (float)(x - m) / mu - (float)m * T;", "float te = (float)(x - m) / mu + (float)m * T;"),
    # likelihood-ratio score of the Poisson arrivals: the -1 dropped
    ("score_poisson", "float g = (float)A / lam - 1.0f;", "float g = (float)A / lam;"),
    # forward scheme: internal arrivals left out of the departure input
    ("forward_missing_ain", "int64_t y = (int64_t)N[i] + A[i] + ain;", "int64_t y = (int64_t)N[i] + A[i];"),
    # arrival integral: sign of the sinusoid term flipped
    ("lambda_sign", "(cos(om * t0 + net->phase) - cos(om * t1 + net->phase))",
     "(cos(om * t1 + net->phase) - cos(om * t0 + net->phase))"),
    # binomial inversion recursion: (n - k) -> (n - k - 1)
    ("binom_inv_recursion", "pk = ((pk * (float)(n - k)) * r) * rinv_tab[k + 1];",
     "pk = ((pk * (float)(n - k - 1)) * r) * rinv_tab[k + 1];"),
    # PTRS constant slip
    ("ptrs_constant", "float a = -0.059f + 0.02483f * b;", "float a = 0.059f + 0.02483f * b;"),
    # BTRS: mode term dropped from the acceptance test
    ("btrs_mode", "if (lv <= logpmf_binom(k, n, p, q) - lpm) return k;",
     "if (lv <= logpmf_binom(k, n, p, q)) return k;"),
    # statistics: busy servers counted as customers
    ("stat_busy", "ss[1] += N[i] < m_t[i] ? N[i] : m_t[i];", "ss[1] += N[i];"),
    # Philox: a Weyl key constant slip
    ("philox_weyl", "#define PHILOX_W1 0xBB67AE85u", "#define PHILOX_W1 0xBB67AE84u"),
    # Lemma 3, m < x <= m + d: exponent x - m written as d
    ("sojourn_lemma3_exponent", "if (x <= m + d) return pow_int(q, x - m) * ((float)(x - d) / (float)m);",
     "if (x <= m + d) return pow_int(q, d) * ((float)(x - d) / (float)m);"),
    # Algorithm 4, backward scheme: post-update count taken as the draw's input
    ("sojourn_backward_x", "const int32_t x = scheme == EO_BACKWARD ? PN(tau, i) : PN(t1, i) + d;",
     "const int32_t x = scheme == EO_BACKWARD ? PN(t1, i) : PN(t1, i) + d;"),
    # Algorithm 4 waiting step: <= m_i written as < m_i
    ("sojourn_wait_threshold", "if (left <= servers_of_step(net, tau + j, dt)[i]) { reached = 1; break; }",
     "if (left < servers_of_step(net, tau + j, dt)[i]) { reached = 1; break; }"),
    # Algorithm 4 routing: departing customer picked with an off-by-one
    ("sojourn_route_pick", "if (k < v) { next = net->col[e]; break; }",
     "if (k <= v) { next = net->col[e]; break; }"),
    # exp: a Taylor coefficient slip
    ("exp_coeff", "p = fmaf(p, r, (float)(1.0 / 6.0));", "p = fmaf(p, r, (float)(1.0 / 7.0));"),
    # resume: the checkpoint ignored (every part restarts from N0)
    ("resume_state_ignored", "N[i] = N_in ? N_in[(int64_t)i * R + r] : net->N0 ? net->N0[i] : 0;",
     "N[i] = net->N0 ? net->N0[i] : 0;"),
    # resume: the checkpoint's own step run again
    ("resume_step_offset", "for (int64_t tau = tau0 + 1; tau <= K && !err; ++tau) {",
     "for (int64_t tau = tau0 > 0 ? tau0 : 1; tau <= K && !err; ++tau) {"),
    # Eq. (1): the busy count not capped at the servers
    ("eq1_busy_uncapped", "    int32_t b = x < m ? x : m;", "    int32_t b = x;"),
    # staffing schedule: a step takes the servers of its end, not its start
    ("staffing_step_end", "int64_t j = (int64_t)floor((double)(tau - 1) * dt / net->sv_dt);",
     "int64_t j = (int64_t)floor((double)tau * dt / net->sv_dt);"),
    # centred gradient estimator: the centring left out
    ("grad_center_ignored", "double x = (g_grad_center ? L - Lbar : L) * sc[r * C + c];",
     "double x = L * sc[r * C + c];"),
    # Algorithm 1's Erlang time drawn from the service stream's own words
    ("erlang_stream_shared", "stream_sibling(&es, st, 2u);", "es = *st;"),
    # coupled gradient: the last step of a perturbation window left unscaled
    ("window_range", "if (tau >= g_win_lo && tau <= g_win_hi) L = L * g_win_factor;",
     "if (tau >= g_win_lo && tau < g_win_hi) L = L * g_win_factor;"),
]


# Slips in the exact DES, which test_oracle_des.py must reject.
DES_MUTANTS = [
    # thinning: every arrival candidate accepted (arrivals at the bound's rate)
    ("des_no_thinning", "if (lmax[i] > 0.0 && rng_u01(&g) * lmax[i] < rate_at(net, i, t)) {",
     "if (lmax[i] > 0.0) {"),
    # service completions at rate N mu instead of min(N, m) mu
    ("des_busy_uncapped", "const int64_t busy = N[i] < m[i] ? N[i] : m[i];\n        srate[i]",
     "const int64_t busy = N[i];\n        srate[i]"),
    # routing ignores the probabilities: always the first edge
    ("des_route_first_edge", "if (v < net->prob[e]) {", "if (v < 2.0) {"),
    # tagged customer: its own completion taken with probability 1 / N, not 1 / busy
    ("des_tag_departure", "} else if (rng_u01(&g) * (double)busy < 1.0) {",
     "} else if (rng_u01(&g) * (double)N[i] < 1.0) {"),
    # tagged customer: a waiting place that never moves up
    ("des_tag_queue", "            tag_pos -= 1;", "            tag_pos -= 0;"),
]

CASES = ([(n, "euler_oracle.c", o, w, "test_oracle_pins.py") for n, o, w in MUTANTS] +
         [(n, "exact_des.c", o, w, "test_oracle_des.py") for n, o, w in DES_MUTANTS])


def _run_mutant(name, target, old, new, suite):
    """Build the oracle with one planted slip and run `suite` against it:
    (returncode, output tail), or (None, message) if the anchor is not unique."""
    src = open(os.path.join(ROOT, "oracle", target)).read()
    if src.count(old) != 1:
        return None, f"mutation anchor for {name} not unique"
    tmp = tempfile.mkdtemp(prefix=f"mut_{name}_")
    try:
        for f in ("euler_oracle.c", "exact_des.c", "euler_oracle.h", "exact_des.h"):
            shutil.copy(os.path.join(ROOT, "oracle", f), tmp)
        with open(os.path.join(tmp, target), "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "liboracle.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", so, os.path.join(tmp, "euler_oracle.c"),
                               os.path.join(tmp, "exact_des.c"), "-lm"])
        env = dict(os.environ, EULER_ORACLE_SO=so, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", suite)],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
        return r.returncode, r.stdout[-2000:]
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.fixture(scope="module")
def mutant_runs():
    """All mutants at once, one process each, as many at a time as there are cores."""
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {c[0]: ex.submit(_run_mutant, *c) for c in CASES}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name,target,old,new,suite", CASES, ids=[c[0] for c in CASES])
def test_pins_reject_mutant(mutant_runs, name, target, old, new, suite):
    rc, out = mutant_runs[name]
    assert rc is not None, out
    assert rc != 0, f"pins did not catch mutant {name}:\n{out}"
