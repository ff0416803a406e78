"""Likelihood-ratio gradients on the GPU: bit-for-bit equal to the CPU
oracle's (per-replication scores, gradient, value, variance; plain and
centred estimators; both launch forms), consistent with central finite
differences under common random numbers, and wired into torch.autograd."""
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


def _queueing_net():
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 0.7)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([6.0, 0.0]), a=1.2, b=0.4, period=3.0, phase=0.5)
    return W.Network(2, row_ptr, col, prob, np.array([2, 3]), np.array([2.5, 1.7]), arr)


def _cases():
    rng = np.random.default_rng(12)
    dag = W.random_small_dag(rng, 9, max_deg=2, m_range=(2, 10), ext_frac=0.7, lam_scale=12.0)
    dag.arrivals.b = 0.5
    return [(_queueing_net(), 0.3, 3.0, 300), (W.tandem3().net, 0.01, 2.0, 100), (dag, 0.05, 2.5, 70)]


@pytest.mark.parametrize("center", [0, 1])
@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("scheme", [0, 1])
def test_grad_matches_oracle_exactly(Bd, orc, case, scheme, form, center):
    """Persistent form (score sums in shared memory) and HBM form (score sums
    per station and replication in global memory) both match the oracle, for
    the plain and the centred estimator."""
    net, dt, T, R = _cases()[case]
    h = Bd.EulerNet(net)
    try:
        h.set_option(Bd.OPT_FORM, form)
        h.set_option(Bd.OPT_GRAD_CENTER, center)
        h.set_option(Bd.OPT_HBM_CHUNK, 64 if center else 0)  # chunked runs too
        g = h.grad(scheme, dt, T, R, 31, rep_begin=5, scores=True, stats=True)
    finally:
        h.close()
    old = orc.set_grad_center(center)
    try:
        want = orc.grad(net, scheme, dt, T, R, 31, rep_begin=5, scores=True)
    finally:
        orc.set_grad_center(old)
    assert np.array_equal(g["scores"].cpu().numpy(), want["scores"])
    assert np.array_equal(g["grad"].cpu().numpy(), want["grad"])
    assert np.array_equal(g["value"].cpu().numpy(), want["value"])
    assert np.array_equal(g["var"].cpu().numpy(), want["var"])
    st = orc.simulate(net, scheme, dt, T, R, 31, rep_begin=5)["stats"]
    assert np.array_equal(g["stats"].cpu().numpy(), st)


def test_grad_full_size_sampled_scores(Bd, orc):
    """The differentiation workload at full size (100-station DAG, sinusoid
    theta = (1, 0.3, 0), 100,000 replications, T = 100, dt = 0.01; the
    planner's form): sampled replications' scores re-run by the oracle match
    bit for bit."""
    run = W.sinusoid_dag()
    h = Bd.EulerNet(run.net)
    try:
        g = h.grad(1, run.dt, run.T, run.R, run.seed, scores=True)
        sc = g["scores"]
        assert bool((g["var"] >= 0).all())
        for r in (0, 4321, run.R - 1):
            want = orc.grad(run.net, 1, run.dt, run.T, 1, run.seed, rep_begin=r, scores=True)["scores"][0]
            assert np.array_equal(sc[r].cpu().numpy(), want)
    finally:
        h.close()


def test_grad_agrees_with_finite_differences(Bd):
    """Central differences under common random numbers (same seed, theta +-
    1e-3 relative) estimate the same derivatives as the likelihood-ratio
    gradient; checked per component within the combined standard errors."""
    import torch
    net = _queueing_net()
    dt, T, R, seed = 0.3, 6.0, 200000, 44
    theta = np.array([*net.mu, net.arrivals.a, net.arrivals.b, net.arrivals.phase])
    h = Bd.EulerNet(net)
    try:
        g = h.grad(1, dt, T, R, seed)
    finally:
        h.close()
    lr, lr_se = g["grad"].cpu().numpy(), np.sqrt(g["var"].cpu().numpy())
    h = Bd.EulerNet(net)
    try:
        h.set_option(Bd.OPT_GRAD_CENTER, 1)
        gc = h.grad(1, dt, T, R, seed)
    finally:
        h.close()
    lrc, lrc_se = gc["grad"].cpu().numpy(), np.sqrt(gc["var"].cpu().numpy())
    assert np.median(lrc_se / lr_se) < 0.5  # the centred estimator's smaller errors
    for c in range(len(theta)):
        d = 1e-3 * max(abs(theta[c]), 0.1)
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[c] += sgn * d
            hh = Bd.EulerNet(Bd._with_theta(net, th))
            try:
                st = hh.simulate(1, dt, T, R, seed).cpu().numpy()
            finally:
                hh.close()
            rp = Bd.split_stats(st, net.n, R)["rep"].astype(np.float64)
            vals.append(np.stack([dt * rp[:, 0], rp[:, 1]]))
        diff = (vals[0] - vals[1]) / (2 * d)  # per replication, CRN
        fd, fd_se = diff.mean(axis=1), diff.std(axis=1) / math.sqrt(R)
        z = (fd - lr[:, c]) / np.sqrt(fd_se ** 2 + lr_se[:, c] ** 2)
        assert np.all(np.abs(z) < 5.0), (c, fd, lr[:, c], z)
        zc = (fd - lrc[:, c]) / np.sqrt(fd_se ** 2 + lrc_se[:, c] ** 2)
        assert np.all(np.abs(zc) < 5.0), (c, fd, lrc[:, c], zc)


def test_autograd_function(Bd):
    import torch
    net = _queueing_net()
    theta = torch.tensor([*net.mu, net.arrivals.a, net.arrivals.b, net.arrivals.phase],
                         dtype=torch.float64, requires_grad=True)
    val = Bd.EulerMeasures.apply(theta, net, 1, 0.3, 3.0, 500, 9)
    (val[0] + 2.0 * val[1]).backward()
    h = Bd.EulerNet(net)
    try:
        g = h.grad(1, 0.3, 3.0, 500, 9)["grad"].cpu().numpy()
    finally:
        h.close()
    assert np.allclose(theta.grad.numpy(), g[0] + 2.0 * g[1], rtol=0, atol=0)
