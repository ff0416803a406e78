"""Likelihood-ratio gradients on the differentiation workload itself: the
100-station DAG with sinusoid arrivals lambda_i(t) = w_i a (1 + b sin(2 pi
t / 24 + phase)), theta = (mu_1..mu_100, a, b, phase), T = 100, dt = 0.01.

* A replication subset at full horizon, in both launch forms, equals the
  oracle's gradient, value, variance and scores bit for bit.
* At full size (100,000 replications) the gradient vector, value and
  variance equal the estimator's definition (blocks of 32 replications,
  ascending, in double) applied to the run's own per-replication scores and
  measures, and sampled replications' scores equal the oracle's: so the whole
  vector is the oracle's estimator.
* Central finite differences at 1e-3 relative under common random numbers
  agree with it for (a, b, phase) and sampled mu_i within the combined
  standard errors.
The gradient has no counterpart in the paper; the estimator is the
likelihood-ratio (score-function) one.
"""
import math

import numpy as np
import pytest

from paper_2402_13259_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Bd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_13259_gb300 import binding
    binding.lib()
    return binding


def _theta(net):
    return np.array([*net.mu, net.arrivals.a, net.arrivals.b, net.arrivals.phase])


@pytest.mark.parametrize("scheme", [0, 1])
def test_c4_subset_matches_oracle(Bd, orc, scheme):
    """32 replications (indices 1000..1031) over the full horizon: the HBM
    form (score sums per station and replication in global memory) and the
    persistent form (in shared memory) both give the oracle's numbers."""
    g = W.sinusoid_dag()
    R, rb = 32, 1000
    h = Bd.EulerNet(g.net)
    got = {}
    try:
        for form in (2, 1):
            h.set_option(Bd.OPT_FORM, form)
            got[form] = h.grad(scheme, g.dt, g.T, R, g.seed, rep_begin=rb, scores=True, stats=True, check=False)
        want = orc.grad(g.net, scheme, g.dt, g.T, R, g.seed, rep_begin=rb, scores=True)
        h.status()
    finally:
        h.close()
    for form, out in got.items():
        for k in ("scores", "grad", "value", "var"):
            a, b = out[k].cpu().numpy(), want[k]
            assert np.array_equal(a, b), (form, k, np.nonzero(a != b))


def _definition(dt, stats, scores, n, R):
    """grad[m][c] = mean_r L_m(r) S_r[c] and the variance of that mean, summed
    in blocks of 32 replications (ascending) then over blocks (ascending)."""
    rp = stats[5 * n: 5 * n + 4 * R].reshape(R, 4)
    L = [dt * rp[:, 0].astype(np.float64), rp[:, 1].astype(np.float64)]
    C = scores.shape[1]
    nb = -(-R // 32)
    grad, var, value = np.zeros((2, C)), np.zeros((2, C)), np.zeros(2)
    for m in range(2):
        x = L[m][:, None] * scores
        pad = np.zeros((nb * 32, C))
        pad[:R] = x
        padL = np.zeros(nb * 32)
        padL[:R] = L[m]
        xb, Lb = pad.reshape(nb, 32, C), padL.reshape(nb, 32)
        part, part2, vpart = np.zeros((nb, C)), np.zeros((nb, C)), np.zeros(nb)
        for k in range(32):
            part = part + xb[:, k, :]
            part2 = part2 + xb[:, k, :] * xb[:, k, :]
            vpart = vpart + Lb[:, k]
        s, ss, vs = np.zeros(C), np.zeros(C), 0.0
        for b in range(nb):
            s = s + part[b]
            ss = ss + part2[b]
            vs = vs + vpart[b]
        value[m] = vs / R
        grad[m] = s / R
        var[m] = (ss - R * grad[m] * grad[m]) / (R * (R - 1.0))
    return grad, value, var


def test_c4_full_size_gradient(Bd, orc):
    """All 100,000 replications, forward scheme, the planner's form."""
    g = W.sinusoid_dag()
    n, R = g.net.n, g.R
    h = Bd.EulerNet(g.net)
    try:
        out = h.grad(1, g.dt, g.T, R, g.seed, scores=True, stats=True, check=False)
        reps = (0, 31, 32, 65536, R - 1)
        want = {r: orc.grad(g.net, 1, g.dt, g.T, 1, g.seed, rep_begin=r, scores=True)["scores"][0] for r in reps}
        h.status()
    finally:
        h.close()
    sc = out["scores"].cpu().numpy()
    st = out["stats"].cpu().numpy()
    for r in reps:
        assert np.array_equal(sc[r], want[r]), r
    grad, value, var = _definition(g.dt, st, sc, n, R)
    assert np.array_equal(out["grad"].cpu().numpy(), grad)
    assert np.array_equal(out["value"].cpu().numpy(), value)
    np.testing.assert_allclose(out["var"].cpu().numpy(), var, rtol=1e-12, atol=0.0)


def test_c4_finite_differences(Bd):
    """Central differences, theta_c +- 1e-3 theta_c (phase: +- 1e-3), same
    seed on both sides (common random numbers), 100,000 replications: the
    per-replication differences estimate the same derivative as the
    likelihood-ratio gradient, within 5 combined standard errors."""
    g = W.sinusoid_dag()
    n, R = g.net.n, g.R
    theta = _theta(g.net)
    h = Bd.EulerNet(g.net)
    try:
        out = h.grad(1, g.dt, g.T, R, g.seed)
    finally:
        h.close()
    lr, lr_se = out["grad"].cpu().numpy(), np.sqrt(out["var"].cpu().numpy())
    params = [n, n + 1, n + 2, 3, 57]  # a, b, phase, mu of a layer-0 and a layer-5 station
    for c in params:
        d = 1e-3 * max(abs(theta[c]), 1.0 if c == n + 2 else 0.0)
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[c] += sgn * d
            hh = Bd.EulerNet(Bd._with_theta(g.net, th))
            try:
                st = hh.simulate(1, g.dt, g.T, R, g.seed).cpu().numpy()
            finally:
                hh.close()
            rp = Bd.split_stats(st, n, R)["rep"].astype(np.float64)
            vals.append(np.stack([g.dt * rp[:, 0], rp[:, 1]]))
        diff = (vals[0] - vals[1]) / (2 * d)
        fd, fd_se = diff.mean(axis=1), diff.std(axis=1) / math.sqrt(R)
        z = (fd - lr[:, c]) / np.sqrt(fd_se ** 2 + lr_se[:, c] ** 2)
        assert np.all(np.abs(z) < 5.0), (c, fd, lr[:, c], z)
