"""Pins of the CPU oracle against facts the paper and mathematics fix.

Each test states what it pins.  A plausible slip in the oracle -- a dropped
term, a wrong branch of Algorithm 1, the backward/forward ordering swapped,
a transposed routing index, a wrong arrival integral -- fails at least one:

* Philox4x32-10 against the published known-answer vectors;
* float math against numpy's double-precision functions (ulp bounds);
* every sampler against its exact law (chi-square / KS, fixed seeds);
* GenerateDeparture (Lemma 1, Algorithm 1) against the exact pure-death
  transition law exp(Q h) of the proof of Lemma 2, by brute force;
* routing against the multinomial pmf (Sec. 2.2);
* the worked 2-node tandem example of Sec. 2.3;
* the infinite-server closed form (Lemma 1(1) + Poisson thinning) of both
  schemes on a random DAG with time-varying arrivals;
* the exact single-station distribution by brute-force convolution;
* Argument 2 and Argument 3 (Sec. 5.1), Theorem 1's steady-state bracketing
  of the Erlang-C mean and gap lambda*h, Theorem 2's per-node gap;
* the arrival integral of Sec. 2.1.1 and the bookkeeping invariants;
* the sojourn sampler of Sec. 6 (Algorithm 4): Lemma 3 against the exact
  tagged-server chain by brute force, and the sojourn law in cases where it is
  known exactly (infinite servers, pure-departure waiting, routing mixture).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm

from paper_2402_13259_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chi2_p(obs, expected, min_exp=10.0):
    obs = np.asarray(obs, dtype=np.float64)
    expected = np.asarray(expected, dtype=np.float64)
    m = expected > min_exp
    # pool everything below the threshold into one cell
    o = np.concatenate([obs[m], [obs[~m].sum()]])
    e = np.concatenate([expected[m], [expected[~m].sum()]])
    keep = e > 0
    o, e = o[keep], e[keep]
    c = ((o - e) ** 2 / e).sum()
    df = max(len(o) - 1, 1)
    return stats.chi2.sf(c, df)


# ---------------------------------------------------------------------------
# Random numbers and float math
# ---------------------------------------------------------------------------
def test_philox_known_answers(orc):
    """Philox4x32-10 reproduces the Random123 known-answer vectors."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split("->")
            v = [int(t, 16) for t in lhs.split()]
            want = [int(t, 16) for t in rhs.split()]
            got = orc.philox(v[:4], v[4:6])
            assert [int(x) for x in got] == want
            n += 1
    assert n == 3


def test_uniform_mapping(orc):
    """Uniforms are odd multiples of 2^-24 in (0,1), built from consecutive
    Philox words of the stream's counter blocks."""
    u = orc.uniforms(seed=0x1234_5678_9ABC, purpose=1, station=7, step=3, rep=11, count=8)
    words = np.concatenate([
        orc.philox([(1 << 24) | b, 7, 3, 11], [0x5678_9ABC, 0x1234]) for b in range(2)])
    want = (((words >> 9) << 1) | 1).astype(np.float64) * 2.0 ** -24
    assert np.array_equal(u.astype(np.float64), want)
    big = orc.uniforms(seed=5, purpose=0, station=0, step=1, rep=0, count=1_000_000)
    assert big.min() >= 2.0 ** -24 and big.max() <= 1 - 2.0 ** -24
    assert abs(big.mean() - 0.5) < 5 * math.sqrt(1 / 12 / big.size)
    assert stats.kstest(big.astype(np.float64), "uniform").pvalue > 1e-4


def _ulps(y, ref):
    sp = np.abs(np.spacing(ref.astype(np.float32))).astype(np.float64)
    return np.abs(y.astype(np.float64) - ref) / sp


def test_float_math_ulp(orc):
    """The oracle's own exp/log/expm1/log1p stay within a few ulp of the
    correctly rounded values (numpy float64 as reference)."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-87, 88.7, 500_000), rng.uniform(-1, 1, 200_000)]).astype(np.float32)
    assert _ulps(orc.map_f32("exp", x), np.exp(x.astype(np.float64))).max() <= 1.0
    x = np.exp(rng.uniform(-87, 88, 500_000)).astype(np.float32)
    x = np.concatenate([x, rng.uniform(0.5, 2.0, 200_000).astype(np.float32)])
    assert _ulps(orc.map_f32("log", x), np.log(x.astype(np.float64))).max() <= 1.0
    x = np.concatenate([rng.uniform(-20, 5, 300_000), -np.exp(rng.uniform(-30, 0, 300_000)),
                        np.exp(rng.uniform(-30, 0, 300_000))]).astype(np.float32)
    assert _ulps(orc.map_f32("expm1", x), np.expm1(x.astype(np.float64))).max() <= 4.0
    x = np.concatenate([rng.uniform(-0.9999, 5, 300_000), -np.exp(rng.uniform(-30, -1e-4, 300_000)),
                        np.exp(rng.uniform(-30, 3, 300_000))]).astype(np.float32)
    assert _ulps(orc.map_f32("log1p", x), np.log1p(x.astype(np.float64))).max() <= 4.0
    special = np.array([0.0, 1.0, -1.0, 100.0, -120.0], dtype=np.float32)
    y = orc.map_f32("exp", special)
    assert y[0] == 1.0 and y[3] == np.inf and y[4] == 0.0
    assert orc.map_f32("log", np.array([1.0], np.float32))[0] == 0.0


# ---------------------------------------------------------------------------
# Samplers against their exact laws
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lam", [1e-3, 0.4, 3.0, 9.99, 10.0, 25.0, 180.0, 5000.0])
def test_poisson_sampler(orc, lam):
    """Poisson(lam): inversion (lam < 10) and PTRS (lam >= 10) follow the pmf."""
    N = 400_000
    x = orc.draw_poisson(lam, 101, N)
    lam32 = float(np.float32(lam))
    hi = int(stats.poisson.isf(1e-9, lam32)) + 2
    obs = np.bincount(x, minlength=hi + 1)
    obs = np.concatenate([obs[:hi], [obs[hi:].sum()]])
    pm = stats.poisson.pmf(np.arange(hi), lam32)
    pm = np.concatenate([pm, [stats.poisson.sf(hi - 1, lam32)]])
    assert _chi2_p(obs, pm * N) > 1e-4
    assert abs(x.mean() - lam32) < 5 * math.sqrt(lam32 / N)


@pytest.mark.parametrize("n,p", [(1, 0.3), (7, 0.3), (100, 0.05), (30, 0.5), (1000, 0.011),
                                 (200, 0.3), (100000, 0.004), (50, 0.9), (700, 0.97),
                                 (2_000_000, 0.45)])
def test_binomial_sampler(orc, n, p):
    """Binomial(n, p): inversion (np < 10), BTRS (np >= 10), symmetric p > 1/2."""
    N = 300_000
    x = orc.draw_binomial(n, p, 202, N)
    p32 = float(np.float32(p))
    lo = int(stats.binom.ppf(1e-9, n, p32))
    hi = int(stats.binom.isf(1e-9, n, p32)) + 1
    ks = np.arange(lo, hi + 1)
    obs = np.bincount(np.clip(x, lo, hi) - lo, minlength=len(ks))
    pm = stats.binom.pmf(ks, n, p32)
    pm[0] = stats.binom.cdf(lo, n, p32)
    pm[-1] = stats.binom.sf(hi - 1, n, p32)
    assert _chi2_p(obs, pm * N) > 1e-4
    assert abs(x.mean() - n * p32) < 5 * math.sqrt(n * p32 * (1 - p32) / N) + 1e-9


def test_binomial_degenerate(orc):
    """Bin(0, p) = 0, Bin(n, 0) = 0, Bin(n, 1) = n (Appendix A's convention)."""
    assert (orc.draw_binomial(0, 0.5, 1, 100) == 0).all()
    assert (orc.draw_binomial(10, 0.0, 1, 100) == 0).all()
    assert (orc.draw_binomial(10, 1.0, 1, 100) == 10).all()


@pytest.mark.parametrize("k", [1, 3, 8, 9, 50, 3000])
def test_erlang_sampler(orc, k):
    """Erlang(k, rate): product-of-uniforms (k <= 8) and Marsaglia-Tsang."""
    g = orc.draw_gamma(k, 2.5, 303, 200_000).astype(np.float64)
    assert stats.kstest(g, stats.gamma(k, scale=1 / 2.5).cdf).pvalue > 1e-4


def test_normal_sampler(orc):
    z = orc.draw_normal(404, 300_000).astype(np.float64)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def _pure_death_law(x, m, mu, h):
    """P(D = d) for the pure departure process from x customers (generator
    q_{y,y-1} = min(y, m) mu, proof of Lemma 2), via the matrix exponential."""
    Q = np.zeros((x + 1, x + 1))
    for y in range(1, x + 1):
        r = min(y, m) * mu
        Q[y, y - 1] = r
        Q[y, y] = -r
    return expm(Q * h)[x][::-1]


@pytest.mark.parametrize("x,m,mu,h", [
    (0, 3, 1.0, 0.5), (5, 8, 1.0, 0.3), (8, 8, 0.7, 0.5), (9, 8, 0.7, 0.5), (12, 3, 2.0, 0.5),
    (40, 3, 1.0, 0.5), (40, 8, 0.5, 2.0), (30, 1, 1.0, 0.05), (25, 4, 3.0, 1.0),
    (60, 5, 0.2, 0.1), (35, 30, 1.0, 0.8)])
def test_departure_exact_law(orc, x, m, mu, h):
    """GenerateDeparture (Algorithm 1) samples the exact law of Lemma 1."""
    N = 400_000
    d = orc.draw_departure(x, m, mu, h, 505, N)
    law = _pure_death_law(x, m, float(np.float32(mu)), float(np.float32(h)))
    obs = np.bincount(d, minlength=x + 1)
    assert d.min() >= 0 and d.max() <= x
    assert _chi2_p(obs, law * N) > 1e-4


def test_route_multinomial(orc):
    """Sequential conditional binomials give Multinomial(D, (p, p_exit))."""
    prob = np.array([0.2, 0.45, 0.15])
    D = 9
    N = 200_000
    out = orc.draw_route(D, prob, 606, N)
    assert (out.sum(axis=1) == D).all() and (out >= 0).all()
    full = np.concatenate([prob, [1 - prob.sum()]])
    keys = out @ np.array([1, 10, 100, 1000])
    uniq, cnt = np.unique(keys, return_counts=True)
    cells = [(u % 10, (u // 10) % 10, (u // 100) % 10, u // 1000) for u in uniq]
    exp = np.array([stats.multinomial.pmf(c, D, full) for c in cells]) * N
    # cells never drawn: their expected mass is the complement
    rest = N - exp.sum()
    assert _chi2_p(np.concatenate([cnt, [0]]), np.concatenate([exp, [max(rest, 0)]])) > 1e-4
    # exit-free row: everything routed, nothing exits
    out2 = orc.draw_route(7, np.array([0.3, 0.7]), 1, 1000)
    assert (out2[:, 2] == 0).all() and (out2[:, :2].sum(axis=1) == 7).all()


# ---------------------------------------------------------------------------
# Schemes
# ---------------------------------------------------------------------------
def _tandem2(mu, servers, lam, dt):
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 1.0)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([lam, 0.0]), a=1.0, b=0.0)
    return W.Network(2, row_ptr, col, prob, np.array(servers), np.array(mu, dtype=float), arr)


def test_worked_example_tandem(orc):
    """Sec. 2.3: one customer arriving in (0, h) with both service times below h
    gives (N_0, N_h, N_2h, N_3h) = (0,1,1,0) backward and (0,0,0,0) forward.
    With mu h = 100 every in-service customer finishes within the step, so the
    schemes are deterministic given the arrivals; replications with exactly
    one arrival in step 1 and none in steps 2-3 realise the example."""
    dt = 0.01
    net = _tandem2([1e4, 1e4], [10, 10], 50.0, dt)
    R = 2000
    b = orc.simulate(net, orc.BACKWARD, dt, 3 * dt, R, 7, trace=True)
    f = orc.simulate(net, orc.FORWARD, dt, 3 * dt, R, 7, trace=True)
    A = b["A"].sum(axis=1)  # [K, R]
    assert np.array_equal(A, f["A"].sum(axis=1))  # common random numbers for arrivals
    sel = (A[0] == 1) & (A[1] == 0) & (A[2] == 0)
    assert sel.sum() > 50
    tb = b["N"].sum(axis=1)[:, sel]
    tf = f["N"].sum(axis=1)[:, sel]
    assert (tb[0] == 1).all() and (tb[1] == 1).all() and (tb[2] == 0).all()
    assert (tf == 0).all()
    # per-node positions in the backward scheme: node 1 at h, node 2 at 2h
    assert (b["N"][0, 0, sel] == 1).all() and (b["N"][1, 1, sel] == 1).all()


def _inf_server_means(net, scheme, dt, K):
    """Exact means when no station ever queues (Lemma 1(1) + thinning):
    backward m_i' = e^{-mu_i h} m_i + L_i + sum_k p_ki (1-e^{-mu_k h}) m_k;
    forward (flow order) y_i = m_i + L_i + sum_k p_ki (1-e^{-mu_k h}) y_k,
    m_i' = e^{-mu_i h} y_i."""
    n = net.n
    a = net.arrivals
    om = 2 * math.pi / a.period
    stay = np.exp(-net.mu * dt)
    m = np.zeros(n) if net.N0 is None else net.N0.astype(float)
    out = np.zeros((K, n))
    for tau in range(1, K + 1):
        t0, t1 = (tau - 1) * dt, tau * dt
        L = a.w * a.a * ((t1 - t0) + a.b * (math.cos(om * t0 + a.phase) - math.cos(om * t1 + a.phase)) / om)
        if scheme == 0:
            new = stay * m + L
            for k in range(n):
                for e in range(net.row_ptr[k], net.row_ptr[k + 1]):
                    new[net.col[e]] += net.prob[e] * (1 - stay[k]) * m[k]
            m = new
        else:
            y = m + L
            for k in range(n):  # stations are numbered in flow order
                for e in range(net.row_ptr[k], net.row_ptr[k + 1]):
                    y[net.col[e]] += net.prob[e] * (1 - stay[k]) * y[k]
            m = stay * y
        out[tau - 1] = m
    return out


@pytest.mark.parametrize("scheme", [0, 1])
def test_infinite_server_closed_form(orc, scheme):
    """With m_i above any reachable count both schemes keep independent Poisson
    counts whose means follow the exact linear recursions above: checks the
    step ordering of Algorithms 2/3, routing indices and arrival integrals."""
    rng = np.random.default_rng(77)
    net = W.random_small_dag(rng, 7, max_deg=3, ext_frac=0.6, lam_scale=20.0)
    net.servers[:] = 1_000_000
    dt, K, R = 0.05, 40, 20000
    res = orc.simulate(net, scheme, dt, K * dt, R, 31, trace=True)
    want = _inf_server_means(net, scheme, dt, K)
    mean = res["N"].mean(axis=2)
    var = res["N"].var(axis=2)
    ok = want > 0.05
    z = (mean[ok] - want[ok]) / np.sqrt(want[ok] / R)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    ratio = (var[ok] / want[ok]).mean()
    assert abs(ratio - 1.0) < 0.02, ratio
    tot = res["N"].sum(axis=1)[-1]
    assert abs(tot.var() / tot.mean() - 1.0) < 0.06


def _single_exact(m, mu, lam, h, N0, K, scheme, smax=90):
    G = np.zeros((smax + 1, smax + 1))
    for x in range(smax + 1):
        law = _pure_death_law(x, m, mu, h)  # P(D = d)
        for d in range(x + 1):
            G[x, x - d] = law[d]
    a = stats.poisson.pmf(np.arange(smax + 1), lam * h)
    P = np.zeros(smax + 1)
    P[N0] = 1.0
    out = []
    for _ in range(K):
        if scheme == 0:
            P = np.convolve(P @ G, a)[: smax + 1]
        else:
            P = np.convolve(P, a)[: smax + 1] @ G
        out.append(P.copy())
    return out


@pytest.mark.parametrize("scheme", [0, 1])
def test_single_station_exact_distribution(orc, scheme):
    """Brute force: backward N_t = G_h(N_{t-1}) + A_t, forward N_t =
    G_h(N_{t-1} + A_t) (Sec. 2.1.3), distribution propagated exactly."""
    m, mu, lam, h, N0, K = 2, 1.0, 3.0, 0.5, 1, 4
    run = W.single_station(m, mu, lam, h, K * h, 200_000, 41, N0=N0)
    res = orc.simulate(run.net, scheme, h, K * h, run.R, run.seed, trace=True)
    exact = _single_exact(m, float(np.float32(mu)), lam, float(np.float32(h)), N0, K, scheme)
    for t in range(K):
        obs = np.bincount(res["N"][t, 0], minlength=91)[:91]
        assert _chi2_p(obs, exact[t] * run.R) > 1e-4


def test_argument3_identity(orc):
    """Argument 3: E[N^b_t] - E[N^f_t] = E[D^f_t] <= m mu h for every t (idle
    start, time-varying arrivals)."""
    m, mu, h, K, R = 5, 1.0, 0.2, 30, 40000
    run = W.single_station(m, mu, 4.0, h, K * h, R, 51, b=0.5, period=3.0)
    b = orc.simulate(run.net, 0, h, K * h, R, 51, trace=True)
    f = orc.simulate(run.net, 1, h, K * h, R, 51, trace=True)
    diff = b["N"][:, 0, :].astype(np.int64) - f["N"][:, 0, :] - f["D"][:, 0, :]
    z = diff.mean(axis=1) / (diff.std(axis=1) / math.sqrt(R) + 1e-12)
    assert np.abs(z).max() < 5.0
    assert (f["D"][:, 0, :].mean(axis=1) <= m * mu * h + 0.02).all()


def test_argument2_identity(orc):
    """Argument 2: N^b_t has the law of N^f_{t-1} + A_t (independent samples)."""
    m, mu, h, K, R = 3, 1.2, 0.3, 12, 60000
    run = W.single_station(m, mu, 3.0, h, K * h, R, 61)
    b = orc.simulate(run.net, 0, h, K * h, R, 61, rep_begin=0, trace=True)
    f = orc.simulate(run.net, 1, h, K * h, R, 61, rep_begin=R, trace=True)
    for t in (1, 4, 11):
        xb = b["N"][t, 0]
        xf = f["N"][t - 1, 0] + f["A"][t, 0]
        top = max(xb.max(), xf.max()) + 1
        cb, cf = np.bincount(xb, minlength=top), np.bincount(xf, minlength=top)
        keep = (cb + cf) > 20
        table = np.stack([np.append(cb[keep], cb[~keep].sum()), np.append(cf[keep], cf[~keep].sum())])
        table = table[:, table.sum(axis=0) > 0]
        assert stats.chi2_contingency(table)[1] > 1e-4


def _erlang_c_mean(m, lam, mu):
    a = lam / mu
    rho = a / m
    top = a ** m / math.factorial(m) / (1 - rho)
    C = top / (sum(a ** k / math.factorial(k) for k in range(m)) + top)
    return a + C * rho / (1 - rho)


def test_steady_state_bracketing(orc):
    """Theorem 1: in steady state N^f <= N <= N^b with E[N^b] - E[N^f] = lambda h;
    E[N] is the Erlang-C mean."""
    m, mu, lam, h = 5, 1.0, 4.0, 0.2
    K, R, burn = 12000, 40, 1000
    run = W.single_station(m, mu, lam, h, K * h, R, 71, N0=7)
    b = orc.simulate(run.net, 0, h, K * h, R, 71, trace=True)["N"][burn:, 0, :].mean(axis=0)
    f = orc.simulate(run.net, 1, h, K * h, R, 71, trace=True)["N"][burn:, 0, :].mean(axis=0)
    EN = _erlang_c_mean(m, lam, mu)
    gap = b - f
    se_gap = gap.std() / math.sqrt(R)
    assert abs(gap.mean() - lam * h) < 5 * se_gap + 0.02
    assert f.mean() < EN < b.mean()
    assert abs((b.mean() + f.mean()) / 2 - EN) < 0.2 * EN


def test_network_steady_state_gap(orc):
    """Theorem 2(i): per node E[N^b(i)] - E[N^f(i)] = lambda~_i h (tandem with
    exits, lambda~ from the traffic equations)."""
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 0.8)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([4.0, 0.0]), a=1.0, b=0.0)
    net = W.Network(2, row_ptr, col, prob, np.array([5, 4]), np.array([1.25, 1.5]), arr,
                    N0=np.array([3, 2]))
    h, K, R, burn = 0.25, 10000, 40, 800
    b = orc.simulate(net, 0, h, K * h, R, 81, trace=True)["N"][burn:].mean(axis=0)
    f = orc.simulate(net, 1, h, K * h, R, 81, trace=True)["N"][burn:].mean(axis=0)
    lam_tot = np.array([4.0, 3.2])
    for i in range(2):
        gap = b[i] - f[i]
        assert abs(gap.mean() - lam_tot[i] * h) < 5 * gap.std() / math.sqrt(R) + 0.02


@pytest.mark.parametrize("kind", ["sinusoid", "table"])
def test_arrival_integral(orc, kind):
    """Sec. 2.1.1: the step's arrival count is Poisson with mean the integral of
    lambda over the step; summed over steps it matches the horizon integral."""
    n = 2
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    if kind == "sinusoid":
        arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([3.0, 7.0]), a=1.5, b=0.6, period=5.0,
                         phase=0.7)
    else:
        tab = np.array([[1.0, 0.0], [4.0, 2.0], [0.5, 6.0], [2.0, 1.0]])
        arr = W.Arrivals(kind=W.ARR_TABLE, table=tab, tab_dt=1.3)
    net = W.Network(n, row_ptr, np.zeros(0), np.zeros(0), np.array([5, 5]), np.array([1.0, 1.0]), arr)
    dt, T, R = 0.07, 6.0, 5000
    res = orc.simulate(net, 0, dt, T, R, 91)
    K = res["K"]
    Tp = K * dt
    if kind == "sinusoid":
        om = 2 * math.pi / arr.period
        want = arr.w * arr.a * (Tp + arr.b * (math.cos(arr.phase) - math.cos(om * Tp + arr.phase)) / om)
    else:
        grid = np.linspace(0.0, Tp, 200001)
        tpts = np.arange(tab.shape[0]) * arr.tab_dt
        want = np.array([np.trapezoid(np.interp(grid, tpts, tab[:, i]), grid) for i in range(n)])
    got = res["station"][:, 4] / R
    assert np.all(np.abs(got - want) < 5 * np.sqrt(want / R))


def test_stats_invariants_and_trace(orc):
    """Stats equal the sums of the traced trajectories; customers are conserved."""
    rng = np.random.default_rng(5)
    net = W.random_small_dag(rng, 9, ext_frac=0.5, lam_scale=8.0)
    net.N0 = rng.integers(0, 6, size=9).astype(np.int32)
    dt, T, R = 0.1, 3.0, 64
    for scheme in (0, 1):
        res = orc.simulate(net, scheme, dt, T, R, 3, trace=True)
        N, D, A = res["N"].astype(np.int64), res["D"].astype(np.int64), res["A"].astype(np.int64)
        st, rp = res["station"], res["rep"]
        assert np.array_equal(st[:, 0], N.sum(axis=(0, 2)))
        assert np.array_equal(st[:, 1], np.minimum(N, net.servers[None, :, None]).sum(axis=(0, 2)))
        assert np.array_equal(st[:, 2], D.sum(axis=(0, 2)))
        assert np.array_equal(st[:, 4], A.sum(axis=(0, 2)))
        assert np.array_equal(rp[:, 0], N.sum(axis=(0, 1)))
        assert np.array_equal(rp[:, 1], D.sum(axis=(0, 1)))
        assert np.array_equal(res["NK"], N[-1].sum(axis=1))
        assert st[:, 3].sum() == rp[:, 2].sum() and st[:, 0].sum() == rp[:, 0].sum()
        total_end = N[-1].sum(axis=0)
        assert np.array_equal(total_end, net.N0.sum() + rp[:, 3] - rp[:, 2])


def test_rep_subsets_are_keyed(orc):
    """Counter-based keying: a replication's results do not depend on which
    batch of replications it is run in (rep_begin offsets)."""
    run = W.tandem3(R=12)
    full = orc.simulate(run.net, 1, run.dt, 2.0, 12, 9)
    a = orc.simulate(run.net, 1, run.dt, 2.0, 5, 9, rep_begin=0)
    b = orc.simulate(run.net, 1, run.dt, 2.0, 7, 9, rep_begin=5)
    assert np.array_equal(full["rep"], np.concatenate([a["rep"], b["rep"]]))
    assert np.array_equal(full["station"], a["station"] + b["station"])


def test_sampler_cap_error_path(orc):
    """A rejection loop that hits its cap reports EO_ERR_SAMPLER_CAP (-5)."""
    run = W.single_station(1000, 1.0, 3000.0, 0.01, 1.0, 50, 1)
    old = orc.set_cap(1)
    try:
        res = orc.simulate(run.net, 0, 0.01, 1.0, 50, 1, expect_ok=False)
    finally:
        orc.set_cap(old)
    assert res["rc"] == -5


def test_validation_errors(orc):
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 0.5), (1, 0, 0.5)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([1.0, 0.0]))
    cyc = W.Network(2, row_ptr, col, prob, np.array([1, 1]), np.array([1.0, 1.0]), arr)
    assert orc.simulate(cyc, 1, 0.1, 1.0, 2, 1, expect_ok=False)["rc"] == -2
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 1.5)])
    bad = W.Network(2, row_ptr, col, prob, np.array([1, 1]), np.array([1.0, 1.0]), arr)
    assert orc.simulate(bad, 0, 0.1, 1.0, 2, 1, expect_ok=False)["rc"] == -1


# ---------------------------------------------------------------------------
# Likelihood-ratio gradients (outside the paper: the paper never
# differentiates; the score terms follow from the laws the method samples)
# ---------------------------------------------------------------------------
def _queueing_net():
    """Two-station tandem with few servers and fast service, so that every
    branch of Algorithm 1 (x <= m, T > h, T <= h) occurs often."""
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 0.7)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([6.0, 0.0]), a=1.2, b=0.4, period=3.0, phase=0.5)
    return W.Network(2, row_ptr, col, prob, np.array([2, 3]), np.array([2.5, 1.7]), arr)


@pytest.mark.parametrize("scheme", [0, 1])
def test_score_has_mean_zero(orc, scheme):
    """E[d log p(path)/d theta] = 0 for every parameter: each per-draw score
    term (binomial in p0(mu), Erlang density, binomial in p(mu, T), Poisson
    in Lambda(a, b, phase)) must be the derivative of its own log-law."""
    net = _queueing_net()
    R = 40000
    orc.counters_reset()
    g = orc.grad(net, scheme, 0.3, 3.0, R, 17, scores=True)
    c = orc.counters()
    assert c["dep_le_m"] > 0 and c["dep_t_gt_h"] > 0 and c["dep_t_le_h"] > 0
    sc = g["scores"]
    z = sc.mean(axis=0) / (sc.std(axis=0) / math.sqrt(R))
    assert np.abs(z).max() < 4.5, z


def _inf_server_measures(net, scheme, dt, K, theta=None, mu=None):
    """Exact E[L1] = dt sum E[N] and E[L2] = sum E[D] when no station queues."""
    import copy
    net2 = copy.deepcopy(net)
    if mu is not None:
        net2.mu = np.asarray(mu, dtype=float)
    if theta is not None:
        net2.arrivals.a, net2.arrivals.b, net2.arrivals.phase = theta
    a = net2.arrivals
    om = 2 * math.pi / a.period
    stay = np.exp(-net2.mu * dt)
    m = np.zeros(net2.n)
    L1 = L2 = 0.0
    for tau in range(1, K + 1):
        t0, t1 = (tau - 1) * dt, tau * dt
        lam = a.w * a.a * ((t1 - t0) + a.b * (math.cos(om * t0 + a.phase) - math.cos(om * t1 + a.phase)) / om)
        if scheme == 0:
            d = (1 - stay) * m
            new = m - d + lam
            for k in range(net2.n):
                for e in range(net2.row_ptr[k], net2.row_ptr[k + 1]):
                    new[net2.col[e]] += net2.prob[e] * d[k]
            m = new
        else:
            y = m + lam
            d = np.zeros(net2.n)
            for k in range(net2.n):
                d[k] = (1 - stay[k]) * y[k]
                for e in range(net2.row_ptr[k], net2.row_ptr[k + 1]):
                    y[net2.col[e]] += net2.prob[e] * d[k]
            m = y - d
        L1 += dt * m.sum()
        L2 += d.sum()
    return np.array([L1, L2])


@pytest.mark.parametrize("scheme", [0, 1])
def test_gradient_matches_infinite_server_closed_form(orc, scheme):
    """With no queueing the means are exact linear recursions; their
    derivatives (central differences of the deterministic recursion) must lie
    inside the LR estimate's confidence interval, for every mu_i and theta."""
    rng = np.random.default_rng(8)
    net = W.random_small_dag(rng, 4, max_deg=2, ext_frac=1.0, lam_scale=8.0)
    net.servers[:] = 1_000_000
    net.arrivals.a, net.arrivals.b, net.arrivals.phase = 1.0, 0.5, 0.3
    dt, K, R = 0.1, 30, 60000
    g = orc.grad(net, scheme, dt, K * dt, R, 23)
    base = _inf_server_measures(net, scheme, dt, K)
    assert np.all(np.abs(g["value"] - base) < 0.02 * base)
    want = np.zeros((2, net.n + 3))
    eps = 1e-5
    for i in range(net.n):
        up, dn = net.mu.copy(), net.mu.copy()
        up[i] += eps
        dn[i] -= eps
        want[:, i] = (_inf_server_measures(net, scheme, dt, K, mu=up) -
                      _inf_server_measures(net, scheme, dt, K, mu=dn)) / (2 * eps)
    th = np.array([net.arrivals.a, net.arrivals.b, net.arrivals.phase])
    for k in range(3):
        up, dn = th.copy(), th.copy()
        up[k] += eps
        dn[k] -= eps
        want[:, net.n + k] = (_inf_server_measures(net, scheme, dt, K, theta=up) -
                              _inf_server_measures(net, scheme, dt, K, theta=dn)) / (2 * eps)
    se = np.sqrt(g["var"])
    z = (g["grad"] - want) / np.maximum(se, 1e-12)
    assert np.abs(z).max() < 5.0, z
    # the centred estimator, mean (L - mean L) S, estimates the same
    # derivatives with smaller standard errors
    old = orc.set_grad_center(1)
    try:
        gc = orc.grad(net, scheme, dt, K * dt, R, 23)
    finally:
        orc.set_grad_center(old)
    assert np.array_equal(gc["value"], g["value"])
    sec = np.sqrt(gc["var"])
    zc = (gc["grad"] - want) / np.maximum(sec, 1e-12)
    assert np.abs(zc).max() < 5.0, zc
    assert (sec <= se).mean() > 0.9 and np.median(sec / np.maximum(se, 1e-300)) < 0.5


# ---------------------------------------------------------------------------
# Average scheme (Sec. 7.1) and step-size rule (Sec. 5.4)
# ---------------------------------------------------------------------------
def test_average_scheme_second_order_on_infinite_server(orc):
    """M/M/inf station: the backward and forward steady states are
    lambda h / (1 - e^{-mu h}) and e^{-mu h} times that (derived from Lemma
    1(1) and the schemes' updates); their average is (lambda/mu)(mu h/2)
    coth(mu h/2) = (lambda/mu)(1 + (mu h)^2/12 + ...), so halving h cuts the
    average's error about four-fold and each scheme's two-fold -- the slope-2
    observation of Sec. 7.3.  The oracle's long-run means follow these forms."""
    lam, mu, R, burn = 40.0, 1.0, 400, 200
    res = {}
    for h in (0.5, 0.25):
        K = int(round(400 / h))
        run = W.single_station(1_000_000, mu, lam, h, K * h, R, 5, N0=40)
        nb = orc.simulate(run.net, 0, h, K * h, R, 5, trace=True)["N"][burn:, 0, :].mean()
        nf = orc.simulate(run.net, 1, h, K * h, R, 5, trace=True)["N"][burn:, 0, :].mean()
        eb = lam * h / (1 - math.exp(-mu * h))
        ef = eb * math.exp(-mu * h)
        assert abs(nb - eb) < 0.01 * eb and abs(nf - ef) < 0.01 * ef
        res[h] = ((nb + nf) / 2 - lam / mu, nb - lam / mu)
    (avg1, b1), (avg2, b2) = res[0.5], res[0.25]
    assert 3.0 < avg1 / avg2 < 5.5, (avg1, avg2)
    assert 1.7 < b1 / b2 < 2.3, (b1, b2)


# ---------------------------------------------------------------------------
# Simpler departure samplers, Eq. (1) and Eq. (2) of Sec. 4.1.1 and 4.1.2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("x,m,mu,h", [(4, 6, 1.0, 0.5), (12, 3, 2.0, 0.5), (30, 8, 0.5, 2.0)])
def test_naive_departure_laws(orc, x, m, mu, h):
    """Eq. (1): D = min(x, Poisson(min(x, m) mu h)); Eq. (2): binomial law of
    Lemma 1(1) for x <= m, Eq. (1) otherwise.  Both over-estimate E[D]
    against the exact law exp(Q h) (the remark after Eq. (1))."""
    N = 300_000
    b = min(x, m)
    lam = float(np.float32(b * float(np.float32(mu * h))))
    pois = stats.poisson.pmf(np.arange(x + 1), lam)
    pois[x] = stats.poisson.sf(x - 1, lam)
    exact = _pure_death_law(x, m, float(np.float32(mu)), float(np.float32(h)))
    old = orc.set_departure_mode(1)
    try:
        d1 = orc.draw_departure(x, m, mu, h, 77, N)
        orc.set_departure_mode(2)
        d2 = orc.draw_departure(x, m, mu, h, 78, N)
    finally:
        orc.set_departure_mode(old)
    assert _chi2_p(np.bincount(d1, minlength=x + 1), pois * N) > 1e-4
    law2 = exact if x <= m else pois
    if x <= m:
        p0 = float(np.float32(-np.expm1(-np.float32(mu * h))))
        law2 = stats.binom.pmf(np.arange(x + 1), x, p0)
    assert _chi2_p(np.bincount(d2, minlength=x + 1), law2 * N) > 1e-4
    e_exact = (exact * np.arange(x + 1)).sum()
    e_naive = (pois * np.arange(x + 1)).sum()
    assert e_naive >= e_exact - 1e-9


# ---------------------------------------------------------------------------
# Time-varying staffing (Sec. 2.1.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", [0, 1])
def test_staffing_schedule_exact_distribution(orc, scheme):
    """With a staffing schedule each step's pure-departure law uses that step's
    servers: the single-station distribution propagated exactly with the
    scheduled m (brute force) matches the oracle; a constant schedule changes
    nothing."""
    mu, lam, h, N0, K = 1.0, 3.0, 0.5, 2, 6
    sched = np.array([[1], [4], [2], [4]], dtype=np.int32)  # m over [0,1), [1,2), [2,3), [3, inf)
    run = W.single_station(4, mu, lam, h, K * h, 200_000, 43, N0=N0)
    net = run.net
    net.servers_schedule, net.servers_schedule_dt = sched, 1.0
    res = orc.simulate(net, scheme, h, K * h, run.R, run.seed, trace=True)
    smax = 90
    a = stats.poisson.pmf(np.arange(smax + 1), lam * h)
    P = np.zeros(smax + 1)
    P[N0] = 1.0
    for t in range(K):
        m = int(sched[min(int((t * h) // 1.0), 3), 0])
        G = np.zeros((smax + 1, smax + 1))
        for x in range(smax + 1):
            law = _pure_death_law(x, m, float(np.float32(mu)), float(np.float32(h)))
            G[x, x - np.arange(x + 1)] = law
        P = np.convolve(P @ G, a)[: smax + 1] if scheme == 0 else np.convolve(P, a)[: smax + 1] @ G
        obs = np.bincount(res["N"][t, 0], minlength=smax + 1)[: smax + 1]
        assert _chi2_p(obs, P * run.R) > 1e-4
    # a constant schedule equal to the servers is the same run
    net2 = W.single_station(4, mu, lam, h, K * h, 500, 43, N0=N0).net
    base = orc.simulate(net2, scheme, h, K * h, 500, 43)["stats"]
    net2.servers_schedule, net2.servers_schedule_dt = np.array([[4]], dtype=np.int32), 1.0
    assert np.array_equal(orc.simulate(net2, scheme, h, K * h, 500, 43)["stats"], base)


# ---------------------------------------------------------------------------
# Sojourn time (Sec. 6, Algorithm 4, Lemma 3)
# ---------------------------------------------------------------------------
def _lemma3_exact(x, m, mu, h):
    """P(tagged server still busy with the same customer | D = d), d = 0..x,
    from the pure departure process with a tagged server: states (y, e), y
    customers left, e = 1 while the tagged customer is still in service."""
    S = 2 * (x + 1)
    Q = np.zeros((S, S))
    for y in range(1, x + 1):
        busy = min(y, m)
        # tagged still in service: its own completion, or one of the others
        Q[2 * y + 1, 2 * (y - 1) + 0] += mu
        Q[2 * y + 1, 2 * (y - 1) + 1] += (busy - 1) * mu
        # tagged gone: every busy server completes at rate mu
        Q[2 * y + 0, 2 * (y - 1) + 0] += busy * mu
    for k in range(S):
        Q[k, k] = -Q[k].sum()
    P = expm(Q * h)[2 * x + 1]
    out = {}
    for d in range(x + 1):
        y = x - d
        tot = P[2 * y] + P[2 * y + 1]
        if tot > 1e-13:
            out[d] = P[2 * y + 1] / tot
    return out


@pytest.mark.parametrize("x,m", [(1, 1), (4, 6), (6, 6), (7, 6), (9, 3), (15, 4), (12, 1), (30, 8)])
@pytest.mark.parametrize("muh", [0.3, 2.0])
def test_sojourn_lemma3_exact(orc, x, m, muh):
    """Lemma 3: the stay probability given the step's departures equals the
    tagged-server chain's conditional probability (and does not depend on mu h)."""
    ex = _lemma3_exact(x, m, 1.0, muh)
    for d, want in ex.items():
        got = orc.sojourn_pstay(x, d, m)
        assert abs(got - want) <= 2e-6 * max(want, 1e-3), (x, m, d, got, want)


def _geom_pmf(p, kmax):
    k = np.arange(1, kmax + 1)
    return (1.0 - p) ** (k - 1) * p


def _p0(mu, h):
    return float(-np.expm1(-np.float64(np.float32(mu * h))))


@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_infinite_server_geometric(orc, scheme):
    """With more servers than customers a customer in service stays through a
    step with probability E[(x - D)/x] = e^{-mu h} for D ~ Bin(x, p0): the
    sojourn in steps is Geometric(p0) exactly, censored at the horizon."""
    mu, h, lam, N0, K, tau0, R = 1.0, 0.05, 400.0, 400, 200, 20, 20000
    run = W.single_station(1_000_000, mu, lam, h, K * h, R, 61, N0=N0)
    res = orc.sojourn(run.net, scheme, h, K * h, R, run.seed, station=0, tau0=tau0)
    s = res["steps"][:, 0]
    kmax = K - tau0
    pmf = _geom_pmf(_p0(mu, h), kmax)
    obs = np.concatenate([np.bincount(s[s > 0], minlength=kmax + 1)[1:], [(s <= 0).sum()]])
    exp_ = np.concatenate([pmf, [1.0 - pmf.sum()]]) * R
    assert s.min() >= -kmax and s.max() <= kmax
    assert _chi2_p(obs, exp_) > 1e-4


@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_waiting_pure_departure(orc, scheme):
    """No arrivals, m servers, the tagged customer last of the p = N_tau0 at
    the station: it reaches a server in the step of the (p - m)-th departure,
    a Gamma(p - m, m mu) time after tau0 h (the paths are exact pure-departure
    paths, Lemma 1), then serves a Geometric(p0) number of steps: S =
    ceil(Gamma / h) + Geometric(p0); S = Geometric(p0) when p <= m."""
    m, mu, h, N0, K, tau0, R = 3, 1.0, 0.02, 12, 1000, 1, 10000
    run = W.single_station(m, mu, 0.0, h, K * h, R, 62, N0=N0)
    res = orc.sojourn(run.net, scheme, h, K * h, R, run.seed, station=0, tau0=tau0)
    s = res["steps"][:, 0]
    # N_tau0 of every path: the first step only (same keys)
    pos = orc.simulate(run.net, scheme, h, tau0 * h, R, run.seed, trace=True)["N"][tau0 - 1, 0]
    hf = float(np.float32(h))
    kmax = K - tau0
    geo = _geom_pmf(_p0(mu, h), kmax)
    mix = np.zeros(kmax)
    for p, cnt in zip(*np.unique(pos, return_counts=True)):
        p = max(int(p), 1)
        if p <= m:
            law = geo
        else:
            F = stats.gamma.cdf(np.arange(0, kmax + 1) * hf, p - m, scale=1.0 / (m * mu))
            eta = np.diff(F)  # P(eta = j), j = 1..kmax
            law = np.convolve(eta, geo)[: kmax]
            law = np.concatenate([[0.0], law[:-1]])  # eta >= 1 then >= 1 service step
        mix += cnt * law
    obs = np.concatenate([np.bincount(s[s > 0], minlength=kmax + 1)[1:], [(s <= 0).sum()]])
    exp_ = np.concatenate([mix, [R - mix.sum()]])
    assert (pos > m).mean() > 0.5  # the waiting step is exercised
    assert _chi2_p(obs, exp_) > 1e-4


@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_heavy_load_service_is_geometric(orc, scheme):
    """A customer that finds a free server (N_tau0 <= m) stays through each
    later step with probability e^{-mu h} whatever the queue behind it: Lemma
    3's x > m branches averaged over the step's departure law.  The load keeps
    x > m in many of those steps."""
    m, mu, lam, h, K, tau0, R = 3, 1.0, 4.5, 0.05, 330, 30, 40000
    run = W.single_station(m, mu, lam, h, K * h, R, 63)
    res = orc.sojourn(run.net, scheme, h, K * h, R, run.seed, station=0, tau0=tau0)
    tr = orc.simulate(run.net, scheme, h, (tau0 + 20) * h, R, run.seed, trace=True)["N"][:, 0]
    sel = tr[tau0 - 1] <= m
    assert sel.mean() > 0.3
    assert (tr[tau0 + 15][sel] > m).mean() > 0.4  # queues behind the customer
    s = res["steps"][sel, 0]
    kmax = K - tau0
    pmf = _geom_pmf(_p0(mu, h), kmax)
    obs = np.concatenate([np.bincount(s[s > 0], minlength=kmax + 1)[1:], [(s <= 0).sum()]])
    exp_ = np.concatenate([pmf, [1.0 - pmf.sum()]]) * sel.sum()
    assert _chi2_p(obs, exp_) > 1e-4


@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_routing_mixture(orc, scheme):
    """Two infinite-server stations, 0 -> 1 with probability p, else exit: the
    customer leaves station 0 to station 1 with probability E[R/D] = p, so S =
    G0 + B G1 with G_i ~ Geometric(p0_i), B ~ Bernoulli(p), independent."""
    p, mu0, mu1, h, K, tau0, R = 0.6, 1.0, 0.25, 0.05, 700, 20, 20000
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, p)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([40.0, 0.0]), a=1.0, b=0.0)
    net = W.Network(2, row_ptr, col, prob, np.full(2, 1_000_000), np.array([mu0, mu1]), arr,
                    N0=np.array([40, 96], dtype=np.int32))
    res = orc.sojourn(net, scheme, h, K * h, R, 64, station=0, tau0=tau0)
    s = res["steps"][:, 0]
    kmax = K - tau0
    g0 = _geom_pmf(_p0(mu0, h), kmax)
    g1 = _geom_pmf(_p0(mu1, h), kmax)
    both = np.concatenate([[0.0], np.convolve(g0, g1)[: kmax - 1]])
    mix = (1.0 - p) * g0 + p * both
    obs = np.concatenate([np.bincount(s[s > 0], minlength=kmax + 1)[1:], [(s <= 0).sum()]])
    exp_ = np.concatenate([mix, [1.0 - mix.sum()]]) * R
    assert _chi2_p(obs, exp_) > 1e-4


def test_sojourn_bookkeeping(orc):
    """Censoring at the horizon, replication keying, the paths' statistics and
    argument errors."""
    run = W.tandem3(R=64)
    net, dt = run.net, run.dt
    K = orc.num_steps(dt, 2.0)
    full = orc.sojourn(net, 0, dt, 2.0, 64, 5, station=0, tau0=50, samples=3)
    assert np.array_equal(full["stats"], orc.simulate(net, 0, dt, 2.0, 64, 5)["stats"])
    sub = orc.sojourn(net, 0, dt, 2.0, 20, 5, station=0, tau0=50, samples=3, rep_begin=30)
    assert np.array_equal(sub["steps"], full["steps"][30:50])
    last = orc.sojourn(net, 1, dt, 2.0, 64, 5, station=1, tau0=K, samples=2)
    assert (last["steps"] == 0).all()  # entered in the last step: censored, nothing accounted
    st = full["steps"]
    assert st.max() <= K - 50 and st.min() >= -(K - 50)
    for bad in (dict(station=3, tau0=1), dict(station=0, tau0=0), dict(station=0, tau0=K + 1)):
        assert orc.sojourn(net, 0, dt, 2.0, 4, 5, expect_ok=False, **bad)["rc"] != 0


# ---------------------------------------------------------------------------
# Checkpoint / resume and the coupled gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", [0, 1])
def test_resume_reproduces_the_uninterrupted_run(orc, scheme):
    """Draws are keyed by (seed, station, step, replication): a run split at
    any steps, each part started from the counts N where the previous one
    stopped, has the statistics of the whole run (sums add up) and its final
    counts, bit for bit."""
    rng = np.random.default_rng(3)
    net = W.random_small_dag(rng, 6, max_deg=2, m_range=(1, 4), ext_frac=0.5, lam_scale=3.0)
    net.N0 = np.arange(6, dtype=np.int32) % 3
    dt, K, R, seed = 0.1, 37, 50, 5
    full = orc.simulate_resume(net, scheme, dt, K * dt, R, seed, 0)
    plain = orc.simulate(net, scheme, dt, K * dt, R, seed)
    assert np.array_equal(full["stats"], plain["stats"])
    for cuts in ([0, 37], [0, 1, 37], [0, 12, 25, 36, 37]):
        st, rp, N = np.zeros_like(full["station"]), np.zeros_like(full["rep"]), None
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = orc.simulate_resume(net, scheme, dt, b * dt, R, seed, a, N)
            st += part["station"]
            rp += part["rep"]
            N = part["N_out"]
            assert np.array_equal(part["NK"], N.sum(axis=1))
        assert np.array_equal(st, full["station"]) and np.array_equal(rp, full["rep"])
        assert np.array_equal(N, full["N_out"])
    # a run with no steps left keeps the checkpoint
    last = orc.simulate_resume(net, scheme, dt, K * dt, R, seed, K, full["N_out"])
    assert np.array_equal(last["N_out"], full["N_out"]) and not last["station"].any()
    # the checkpoint is per replication: other counts give another continuation
    other = orc.simulate_resume(net, scheme, dt, K * dt, R, seed, 12, np.zeros((6, R), np.int32))
    assert not np.array_equal(other["N_out"], full["N_out"])


def _inf_server_measures_scaled(net, scheme, dt, K, scale):
    """E[L1], E[L2] of the no-queueing recursion with Lambda_tau scaled by scale(tau)."""
    a = net.arrivals
    om = 2 * math.pi / a.period
    stay = np.exp(-net.mu * dt)
    m = np.zeros(net.n)
    L1 = L2 = 0.0
    for tau in range(1, K + 1):
        t0, t1 = (tau - 1) * dt, tau * dt
        lam = scale(tau) * a.w * a.a * ((t1 - t0) + a.b * (math.cos(om * t0 + a.phase) - math.cos(om * t1 + a.phase)) / om)
        if scheme == 0:
            d = (1 - stay) * m
            new = m - d + lam
            for k in range(net.n):
                for e in range(net.row_ptr[k], net.row_ptr[k + 1]):
                    new[net.col[e]] += net.prob[e] * d[k]
            m = new
        else:
            y = m + lam
            d = np.zeros(net.n)
            for k in range(net.n):
                d[k] = (1 - stay[k]) * y[k]
                for e in range(net.row_ptr[k], net.row_ptr[k + 1]):
                    y[net.col[e]] += net.prob[e] * d[k]
            m = y - d
        L1 += dt * m.sum()
        L2 += d.sum()
    return np.array([L1, L2])


@pytest.mark.parametrize("scheme", [0, 1])
def test_coupled_gradient_infinite_server_closed_form(orc, scheme):
    """Without queueing E[L] follows exact linear recursions, so the expected
    central difference of each parameter (mu_i at mu_i (1 +- delta); the
    arrival means of one time window at (1 +- delta)) is known: the coupled
    estimator must match it within its confidence interval.  Its window
    derivatives add up to the derivative for scaling every step, the
    integral of the response to an arrival over the rest of the horizon."""
    rng = np.random.default_rng(8)
    net = W.random_small_dag(rng, 4, max_deg=2, ext_frac=1.0, lam_scale=8.0)
    net.servers[:] = 1_000_000
    net.arrivals.a, net.arrivals.b, net.arrivals.phase = 1.0, 0.5, 0.3
    dt, K, R, W_, delta = 0.1, 30, 4000, 3, 0.05
    g = orc.grad_coupled(net, scheme, dt, K * dt, R, 23, W_, delta)
    want = np.zeros((2, net.n + W_))
    for i in range(net.n):
        up, dn = net.mu.copy(), net.mu.copy()
        up[i] *= 1 + delta
        dn[i] *= 1 - delta
        want[:, i] = (_inf_server_measures(net, scheme, dt, K, mu=up) -
                      _inf_server_measures(net, scheme, dt, K, mu=dn)) / (2 * delta * net.mu[i])
    for w in range(W_):
        lo, hi = w * K // W_ + 1, (w + 1) * K // W_
        f = lambda s: (lambda tau: s if lo <= tau <= hi else 1.0)  # noqa: E731
        want[:, net.n + w] = (_inf_server_measures_scaled(net, scheme, dt, K, f(1 + delta)) -
                              _inf_server_measures_scaled(net, scheme, dt, K, f(1 - delta))) / (2 * delta)
    se = np.sqrt(g["var"])
    z = (g["grad"] - want) / np.maximum(se, 1e-12)
    assert np.abs(z).max() < 5.0, z
    # linear in the arrival scale: the windows add up to the whole horizon's
    whole = (_inf_server_measures_scaled(net, scheme, dt, K, lambda t: 1 + delta) -
             _inf_server_measures_scaled(net, scheme, dt, K, lambda t: 1 - delta)) / (2 * delta)
    assert np.allclose(want[:, net.n:].sum(axis=1), whole, rtol=1e-9)
    # a later window matters less for the time-integrated count (less time left)
    assert want[0, net.n] > want[0, net.n + 1] > want[0, net.n + 2] > 0


@pytest.mark.parametrize("scheme", [0, 1])
def test_coupled_gradient_agrees_with_likelihood_ratio(orc, scheme):
    """On a queueing tandem where every branch of Algorithm 1 occurs, the
    coupled central differences in mu_i and the likelihood-ratio gradient
    estimate the same derivatives (up to the O(delta^2) bias of a central
    difference).  Common random numbers keep the two runs' paths together:
    the per-replication spread of the difference quotient is well below
    that of the same quotient from independent runs,
    sqrt(2 Var L) / (2 delta mu)."""
    net = _queueing_net()
    dt, T, R, Rc, delta = 0.3, 3.0, 40000, 4000, 0.05
    old = orc.set_grad_center(1)
    try:
        lr = orc.grad(net, scheme, dt, T, R, 17)
    finally:
        orc.set_grad_center(old)
    cp = orc.grad_coupled(net, scheme, dt, T, Rc, 17, 2, delta, params=[0, 1])
    se = np.sqrt(lr["var"][:, :2] + cp["var"])
    z = (cp["grad"] - lr["grad"][:, :2]) / se
    assert np.abs(z).max() < 5.0, z
    base = orc.simulate(net, scheme, dt, T, Rc, 17)
    L = [dt * base["rep"][:, 0], base["rep"][:, 1]]
    independent = np.array([[math.sqrt(2 * L[m].var()) / (2 * delta * net.mu[c]) for c in (0, 1)]
                            for m in (0, 1)])
    coupled = np.sqrt(cp["var"] * Rc)
    ratio = coupled / independent
    assert np.all(ratio < 0.5) and np.median(ratio) < 0.2, ratio


@pytest.mark.parametrize("scheme", [0, 1])
def test_coupled_windows_add_up_to_the_arrival_scale(orc, scheme):
    """On the queueing tandem, scaling the arrival means of every step by s
    is scaling the sinusoid's amplitude a, so the coupled window derivatives
    summed over the windows estimate a dL/da, which the likelihood-ratio
    gradient estimates independently (to first order in delta: the windows'
    central differences interact only at O(delta^2))."""
    net = _queueing_net()
    dt, T, R, Rc, W_, delta = 0.3, 3.0, 40000, 4000, 3, 0.05
    old = orc.set_grad_center(1)
    try:
        lr = orc.grad(net, scheme, dt, T, R, 29)
    finally:
        orc.set_grad_center(old)
    cp = orc.grad_coupled(net, scheme, dt, T, Rc, 29, W_, delta, params=[net.n + w for w in range(W_)])
    a = net.arrivals.a
    want = a * lr["grad"][:, net.n]
    got = cp["grad"].sum(axis=1)
    se = np.sqrt(a * a * lr["var"][:, net.n] + cp["var"].sum(axis=1))
    assert np.all(np.abs(got - want) < 5.0 * se + 0.02 * np.abs(want)), (got, want, se)
    assert np.all(got > 0)  # more arrivals: more customers and more departures
