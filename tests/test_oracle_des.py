"""The exact DES (oracle/exact_des.c) pinned to closed forms, then used to
check properties the paper proves for the Euler schemes.

DES pins: M(t)/M/inf transient law with sinusoidal arrivals (thinning), the
Erlang-C stationary law of M/M/c, the Jackson product form of a stationary
tandem, and the transient law of a tiny network by brute-force matrix
exponential.  Properties of the schemes against the DES: the backward and
forward means bracket the exact means (Argument 1 for a single station at
every step; Theorem 2 at every node of a network in steady state, with the
gap lambda~_i h), the stationary gap of Theorem 1, and the error's decay as h
shrinks (Theorem 1, Sec. 7.3) and as the system grows at fixed h (Sec. 5.3).
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm

from paper_2402_13259_gb300 import workloads as W


def _chi2_p(obs, expected, min_exp=10.0):
    obs = np.asarray(obs, dtype=np.float64)
    expected = np.asarray(expected, dtype=np.float64)
    m = expected > min_exp
    o = np.concatenate([obs[m], [obs[~m].sum()]])
    e = np.concatenate([expected[m], [expected[~m].sum()]])
    keep = e > 0
    o, e = o[keep], e[keep]
    return stats.chi2.sf(((o - e) ** 2 / e).sum(), max(len(o) - 1, 1))


def _mmc_pmf(lam, mu, c, kmax):
    """Stationary M/M/c law P(N = k), k = 0..kmax."""
    a = lam / mu
    rho = a / c
    w = np.array([a ** k / math.factorial(k) if k <= c else
                  a ** c / math.factorial(c) * rho ** (k - c) for k in range(kmax + 1)])
    tail = a ** c / math.factorial(c) * rho ** (kmax + 1 - c) / (1.0 - rho)  # k > kmax
    return w / (w.sum() + tail)


def _erlang_c_mean(lam, mu, c):
    a = lam / mu
    rho = a / c
    s = sum(a ** k / math.factorial(k) for k in range(c))
    top = a ** c / math.factorial(c) / (1.0 - rho)
    pw = top / (s + top)
    return pw * rho / (1.0 - rho) + a


def test_des_mminf_sinusoid_transient(orc):
    """M(t)/M/inf from empty: N(t) ~ Poisson(M(t)), M(t) = int_0^t lambda(s)
    e^{-mu (t-s)} ds in closed form for lambda(s) = w (1 + b sin(om s + ph))."""
    w, b, period, mu, dt, K, R = 40.0, 0.6, 6.0, 1.3, 0.5, 12, 20000
    run = W.single_station(10 ** 6, mu, w, dt, K * dt, R, 7, b=b, period=period)
    run.net.arrivals.phase = 0.4
    ph = 0.4
    res = orc.des_simulate(run.net, dt, K * dt, R, 7, trace=True)
    om = 2 * math.pi / period
    for k in range(1, K + 1):
        t = k * dt
        integ = ((mu * math.sin(om * t + ph) - om * math.cos(om * t + ph))
                 - math.exp(-mu * t) * (mu * math.sin(ph) - om * math.cos(ph))) / (mu * mu + om * om)
        M = w / mu * (1 - math.exp(-mu * t)) + w * b * integ
        x = res["N"][k - 1, 0]
        assert abs(x.mean() - M) < 5 * math.sqrt(M / R), (k, x.mean(), M)
        assert abs(x.var() / M - 1.0) < 0.06
        if k in (4, 12):
            kk = np.arange(0, int(M + 8 * math.sqrt(M)) + 1)
            assert _chi2_p(np.bincount(x, minlength=len(kk))[:len(kk)], stats.poisson.pmf(kk, M) * R) > 1e-4


def test_des_erlang_c_stationary(orc):
    """M/M/c started near equilibrium: at a late time the count follows the
    stationary M/M/c law, whose mean is the Erlang-C formula."""
    lam, mu, c, R = 2.4, 1.0, 3, 30000
    run = W.single_station(c, mu, lam, 1.0, 40.0, R, 11, N0=3)
    res = orc.des_simulate(run.net, 1.0, 40.0, R, 11, trace=True)
    x = res["N"][-1, 0]
    kmax = 40
    pmf = _mmc_pmf(lam, mu, c, kmax)
    assert _chi2_p(np.bincount(np.minimum(x, kmax + 1), minlength=kmax + 2)[:kmax + 1], pmf * R) > 1e-4
    L = _erlang_c_mean(lam, mu, c)
    assert abs(x.mean() - L) < 5 * x.std() / math.sqrt(R)


def test_des_jackson_tandem(orc):
    """Stationary tandem M/M/2 -> M/M/3: the joint law is the product of the
    two M/M/c marginals (Jackson)."""
    lam, mu1, mu2, R = 1.5, 1.0, 0.8, 20000
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 1.0)])
    net = W.Network(2, row_ptr, col, prob, np.array([2, 3]), np.array([mu1, mu2]),
                    W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([lam, 0.0]), a=1.0, b=0.0),
                    N0=np.array([2, 2], dtype=np.int32))
    res = orc.des_simulate(net, 1.0, 60.0, R, 13, trace=True)
    n1, n2 = res["N"][-1, 0], res["N"][-1, 1]
    k = 12
    p1, p2 = _mmc_pmf(lam, mu1, 2, k), _mmc_pmf(lam, mu2, 3, k)
    joint = np.outer(p1, p2)
    obs = np.zeros((k + 1, k + 1))
    ok = (n1 <= k) & (n2 <= k)
    np.add.at(obs, (n1[ok], n2[ok]), 1)
    assert _chi2_p(obs.ravel(), joint.ravel() * R) > 1e-4
    assert abs(np.corrcoef(n1, n2)[0, 1]) < 0.03


def test_des_brute_force_transient(orc):
    """A 2-station network from (2, 0): the law of (N_0, N_1) at t = 1.5 by
    the matrix exponential of the (truncated) generator."""
    lam, mu, m, p01, t, R = 0.9, (1.3, 0.7), (1, 2), 0.6, 1.5, 40000
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, p01)])
    net = W.Network(2, row_ptr, col, prob, np.array(m), np.array(mu),
                    W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([lam, 0.0]), a=1.0, b=0.0),
                    N0=np.array([2, 0], dtype=np.int32))
    cap = 22
    idx = lambda a, b: a * (cap + 1) + b  # noqa: E731
    S = (cap + 1) ** 2
    Q = np.zeros((S, S))
    for a in range(cap + 1):
        for b in range(cap + 1):
            s = idx(a, b)
            if a < cap:
                Q[s, idx(a + 1, b)] += lam
            if a > 0:
                r = min(a, m[0]) * mu[0]
                if b < cap:
                    Q[s, idx(a - 1, b + 1)] += r * p01
                Q[s, idx(a - 1, b)] += r * (1 - p01)
            if b > 0:
                Q[s, idx(a, b - 1)] += min(b, m[1]) * mu[1]
    Q -= np.diag(Q.sum(axis=1))
    P = expm(Q * t)[idx(2, 0)].reshape(cap + 1, cap + 1)
    res = orc.des_simulate(net, t, t, R, 17, trace=True)
    n0, n1 = res["N"][0, 0], res["N"][0, 1]
    obs = np.zeros((cap + 1, cap + 1))
    np.add.at(obs, (np.minimum(n0, cap), np.minimum(n1, cap)), 1)
    assert _chi2_p(obs.ravel(), P.ravel() * R) > 1e-4


def test_des_bookkeeping(orc):
    """Departures, exits and arrivals balance; the statistics match the trace;
    replication subsets are keyed; staffing schedules run."""
    run = W.tandem3(R=30)
    d = orc.des_simulate(run.net, run.dt, 3.0, 30, 5, trace=True)
    st, rp = d["station"], d["rep"]
    assert st[:, 0].sum() == rp[:, 0].sum() == d["N"].sum()
    assert d["NK"].sum() == rp[:, 3].sum() - rp[:, 2].sum()
    assert (st[:, 1] <= st[:, 0]).all()
    sub = orc.des_simulate(run.net, run.dt, 3.0, 10, 5, rep_begin=20)
    assert np.array_equal(sub["rep"], rp[20:30])
    net = run.net
    net.servers_schedule = np.array([[50, 50, 50], [5, 8, 50]], dtype=np.int32)
    net.servers_schedule_dt = 1.5
    s = orc.des_simulate(net, run.dt, 3.0, 30, 5)
    assert s["station"][0, 0] > st[0, 0]  # fewer servers after t = 1.5: longer queues


# ---------------------------------------------------------------------------
# The Euler schemes against the exact process
# ---------------------------------------------------------------------------
def _means(res, R):
    return res["N"].mean(axis=2), res["N"].std(axis=2) / math.sqrt(R)


def test_single_station_bracketing_transient(orc):
    """Argument 1 (Sec. 5.1): for a single station N^f_tau <= N_tau <= N^b_tau
    in distribution at every tau, here with time-varying arrivals from an
    empty start: the means are ordered at every observation time."""
    run = W.single_station(6, 1.0, 5.0, 0.1, 6.0, 6000, 3, b=0.5, period=3.0)
    net, dt, T, R = run.net, 0.1, 6.0, 6000
    e = orc.des_simulate(net, dt, T, R, 21, trace=True)
    b = orc.simulate(net, 0, dt, T, R, 22, trace=True)
    f = orc.simulate(net, 1, dt, T, R, 23, trace=True)
    me, se = _means(e, R)
    mb, sb = _means(b, R)
    mf, sf = _means(f, R)
    tol = 4.5 * np.sqrt(se ** 2 + np.maximum(sb, sf) ** 2) + 1e-9
    assert (mf <= me + tol).all() and (me <= mb + tol).all()
    assert (mb - mf).mean() > 0.2


def _traffic(net, lam):
    """Total arrival rates lambda~ = lambda + P^T lambda~ (Theorem 2)."""
    n = net.n
    P = np.zeros((n, n))
    for i in range(n):
        for e in range(net.row_ptr[i], net.row_ptr[i + 1]):
            P[i, net.col[e]] += net.prob[e]
    return np.linalg.solve(np.eye(n) - P.T, lam)


@pytest.mark.parametrize("case", ["tandem", "dag"])
def test_network_steady_state_bracketing_and_gap(orc, case):
    """Theorem 2 (i): in steady state N^f(i) <= N(i) <= N^b(i) at every node,
    with E[N^b(i)] - E[N^f(i)] = lambda~_i h.  (Transiently the order can fail
    at downstream nodes, as Sec. 5.2 notes; the means here are taken after a
    burn-in.)"""
    h = 0.1
    if case == "tandem":
        row_ptr, col, prob = W.csr_from_edges(3, [(0, 1, 1.0), (1, 2, 0.7)])
        lam = np.array([4.0, 0.0, 1.0])
        net = W.Network(3, row_ptr, col, prob, np.array([5, 6, 6]), np.array([1.0, 0.9, 1.1]),
                        W.Arrivals(kind=W.ARR_SINUSOID, w=lam, a=1.0, b=0.0),
                        N0=np.array([4, 4, 4], dtype=np.int32))
    else:
        rng = np.random.default_rng(5)
        net = W.random_small_dag(rng, 6, max_deg=2, m_range=(3, 8), ext_frac=0.5, lam_scale=1.0)
        tot = _traffic(net, net.arrivals.w)
        net.servers = np.maximum(net.servers, np.ceil(tot / (0.8 * net.mu))).astype(np.int32)
        lam = net.arrivals.w
    T, R, kb = 40.0, 2000, 100
    e = orc.des_simulate(net, h, T, R, 21, trace=True)["N"][kb:]
    b = orc.simulate(net, 0, h, T, R, 22, trace=True)["N"][kb:]
    f = orc.simulate(net, 1, h, T, R, 23, trace=True)["N"][kb:]
    tot = _traffic(net, np.asarray(lam, dtype=float))
    assert (tot > 0).sum() >= 3
    for i in range(net.n):
        if tot[i] <= 0:
            continue  # a node no customer reaches
        # replication means are independent; the time average inside one is not
        ve, vb, vf = (x[:, i, :].mean(axis=0) for x in (e, b, f))
        se = math.sqrt((ve.var() + max(vb.var(), vf.var())) / R)
        assert vf.mean() <= ve.mean() + 4.5 * se and ve.mean() <= vb.mean() + 4.5 * se, i
        gap = vb.mean() - vf.mean()
        assert abs(gap - tot[i] * h) < 4.5 * math.sqrt((vb.var() + vf.var()) / R) + 0.03 * tot[i] * h, (i, gap, tot[i] * h)


def test_stationary_gap_and_error_decay_in_h(orc):
    """Single M/M/c station in steady state: backward above, forward below
    the exact (Erlang-C) mean, the gap equal to lambda h (Theorem 1), and the
    error of each scheme shrinking with h.  (How the gap splits between the
    two is not fixed by the theorem: here the backward scheme is much closer,
    so their average is not the better estimate at these h.)"""
    lam, mu, c = 4.0, 1.0, 5
    L = _erlang_c_mean(lam, mu, c)
    errs = {}
    for h in (0.2, 0.1, 0.05):
        T, R, burn = 60.0, 3000, 20.0
        K, kb = int(round(T / h)), int(round(burn / h))
        run = W.single_station(c, mu, lam, h, T, R, 31, N0=4)
        b = orc.simulate(run.net, 0, h, T, R, 32, trace=True)
        f = orc.simulate(run.net, 1, h, T, R, 33, trace=True)
        nb, nf, df = b["N"][kb:, 0], f["N"][kb:, 0], f["D"][kb:, 0]
        mb, mf = nb.mean(), nf.mean()
        assert mf < L < mb
        # Argument 1: E[N_tau^b] - E[N_tau^f] = E[D_tau^f] at every tau (same N_0), and
        # in steady state E[D^f] = lambda h.  Replications are independent, the time
        # average inside one is not: the standard error comes from replication means.
        rb, rf, rd = nb.mean(axis=0), nf.mean(axis=0), df.mean(axis=0)
        se = math.sqrt((rb.var() + np.var(rf - rd)) / R)
        assert abs((mb - mf) - df.mean()) < 4.5 * se, (h, mb - mf, df.mean(), se)
        assert abs(df.mean() - lam * h) < 0.03 * lam * h
        errs[h] = (mb - L, L - mf, abs(0.5 * (mb + mf) - L))
    assert errs[0.05][0] < 0.7 * errs[0.2][0] and errs[0.05][1] < 0.7 * errs[0.2][1]


def test_relative_error_under_the_selection_rule(orc):
    """Sec. 5.3 / Theorem 3: in steady state RE^b + RE^f = lambda h / E[N] <=
    mu h (relative errors against the exact Erlang-C mean); with h from the
    selection rule h = alpha_m / mu, alpha_m = 0.4 / sqrt(m) (Sec. 5.4, Sec.
    7.4), the relative error shrinks as the station grows (same utilisation)."""
    mu, rho = 1.0, 0.8
    total = []
    for c, T, burn in ((4, 150.0, 50.0), (64, 60.0, 10.0)):
        lam = rho * c * mu
        h = 0.4 / math.sqrt(c) / mu
        L = _erlang_c_mean(lam, mu, c)
        R, kb = 1000, int(round(burn / h))
        run = W.single_station(c, mu, lam, h, T, R, 41, N0=int(round(L)))
        mb = orc.simulate(run.net, 0, h, T, R, 42, trace=True)["N"][kb:, 0].mean(axis=0)
        mf = orc.simulate(run.net, 1, h, T, R, 43, trace=True)["N"][kb:, 0].mean(axis=0)
        re_b, re_f = (mb.mean() - L) / L, (L - mf.mean()) / L
        se = math.sqrt(mb.var() / R + mf.var() / R) / L
        bound = lam * h / L
        assert abs((re_b + re_f) - bound) < 4.5 * se + 0.02 * bound, (c, re_b, re_f, bound)
        assert re_b < mu * h + 4.5 * se and re_f < mu * h + 4.5 * se
        total.append(re_b + re_f)
    assert total[1] < 0.6 * total[0]


def test_des_sojourn_exact_laws(orc):
    """The DES's tagged customer: in a stationary FCFS M/M/1 queue an arriving
    customer's sojourn is Exp(mu - lambda) (PASTA); through two infinite-server
    stations with a routing split it is Exp(mu_1) plus, with probability p,
    an independent Exp(mu_2)."""
    lam, mu, R = 0.7, 1.0, 20000
    run = W.single_station(1, mu, lam, 1.0, 200.0, R, 3, N0=2)
    t = orc.des_sojourn(run.net, 1.0, 200.0, R, 9, 0, 60.0)
    assert (t < 0).sum() == 0
    assert stats.kstest(t, stats.expon(scale=1.0 / (mu - lam)).cdf).pvalue > 1e-4
    p, mu1, mu2 = 0.4, 2.0, 0.5
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, p)])
    net = W.Network(2, row_ptr, col, prob, np.full(2, 10 ** 6), np.array([mu1, mu2]),
                    W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([5.0, 0.0]), a=1.0, b=0.0))
    t = orc.des_sojourn(net, 1.0, 200.0, R, 11, 0, 3.0)
    x = np.linspace(0.05, 12, 40)
    # P(T <= x) for the mixture (1-p) Exp(mu1) + p (Exp(mu1) + Exp(mu2))
    hypo = (1 - p) * (1 - np.exp(-mu1 * x)) + p * (1 - (mu1 * np.exp(-mu2 * x) - mu2 * np.exp(-mu1 * x)) / (mu1 - mu2))
    emp = (t[None, :] <= x[:, None]).mean(axis=1)
    assert np.abs(emp - hypo).max() < 1.36 * 1.3 / math.sqrt(R) * 3, np.abs(emp - hypo).max()


def test_sojourn_converges_to_exact(orc):
    """Sec. 7.6: the sojourn-time law of Algorithm 4 approaches the exact one
    (a tagged customer followed through the DES under FCFS) as h shrinks: the
    KS distance and the error of the mean fall from h = 0.2 to h = 0.05."""
    run = W.tandem3()
    T, t0, R = 20.0, 5.0, 6000
    d = orc.des_sojourn(run.net, 0.05, T, R, 7, 0, t0)
    assert (d < 0).mean() < 0.002  # (nearly) every tagged customer left by T
    se = d.std() / math.sqrt(R)
    for scheme in (0, 1):
        err, ks = {}, {}
        for h in (0.2, 0.05):
            e = orc.sojourn(run.net, scheme, h, T, R, 8, 0, int(round(t0 / h)))["steps"][:, 0] * h
            err[h] = abs(e.mean() - d.mean())
            ks[h] = stats.ks_2samp(e, d).statistic
        assert ks[0.05] < 0.6 * ks[0.2] and ks[0.05] < 0.06, (scheme, ks)
        assert err[0.05] < 0.5 * err[0.2] + 3 * se and err[0.05] < 0.1 + 4 * se, (scheme, err)
