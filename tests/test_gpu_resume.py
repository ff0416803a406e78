"""Checkpoint / resume and the coupled (common-random-numbers) gradient with
checkpointed replay on the GPU: bit for bit the oracle's, on small cases
(ragged replication counts, chunked runs, both schemes), and the split-run
property at the benchmark's size."""
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


def _net():
    rng = np.random.default_rng(3)
    net = W.random_small_dag(rng, 6, max_deg=2, m_range=(1, 4), ext_frac=0.5, lam_scale=3.0)
    net.N0 = (np.arange(6) % 3).astype(np.int32)
    return net


def _queueing_net():
    row_ptr, col, prob = W.csr_from_edges(2, [(0, 1, 0.7)])
    arr = W.Arrivals(kind=W.ARR_SINUSOID, w=np.array([6.0, 0.0]), a=1.2, b=0.4, period=3.0, phase=0.5)
    return W.Network(2, row_ptr, col, prob, np.array([2, 3]), np.array([2.5, 1.7]), arr)


@pytest.mark.parametrize("chunk", [0, 32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_resume_matches_oracle(Bd, orc, scheme, chunk):
    """Each part of a run split at steps 12 and 25 equals the oracle's part
    (statistics and N at the cut), the parts add up to the whole run, and the
    whole equals euler_net_simulate in the planner's own form."""
    net = _net()
    dt, K, R, seed = 0.1, 37, 100, 5
    h = Bd.EulerNet(net)
    try:
        if chunk:
            h.set_option(Bd.OPT_HBM_CHUNK, chunk)
        N = None
        Nd = None
        tot = np.zeros(Bd.stats_len(net.n, R), dtype=np.int64)
        for a, b in ((0, 12), (12, 25), (25, K)):
            st, Nout = h.simulate_resume(scheme, dt, b * dt, R, seed, a, state_in=Nd, state_out=True,
                                         rep_begin=7)
            want = orc.simulate_resume(net, scheme, dt, b * dt, R, seed, a, N, rep_begin=7)
            assert np.array_equal(st.cpu().numpy(), want["stats"]), (a, b)
            assert np.array_equal(Nout.cpu().numpy(), want["N_out"]), (a, b)
            N, Nd = want["N_out"], Nout
            s = st.cpu().numpy()
            tot[: 5 * net.n + 4 * R] += s[: 5 * net.n + 4 * R]
            tot[5 * net.n + 4 * R:] = s[5 * net.n + 4 * R:]
        whole = h.simulate(scheme, dt, K * dt, R, seed, rep_begin=7).cpu().numpy()
        assert np.array_equal(tot, whole)
        # no steps left: the checkpoint comes back, nothing is counted
        st, Nout = h.simulate_resume(scheme, dt, K * dt, R, seed, K, state_in=Nd, state_out=True,
                                     rep_begin=7)
        s = st.cpu().numpy()
        assert np.array_equal(Nout.cpu().numpy(), N) and not s[: 5 * net.n + 4 * R].any()
        assert np.array_equal(s[5 * net.n + 4 * R:], N.sum(axis=1))
        # a bad step_begin is refused synchronously
        with pytest.raises(Bd.EulerError):
            h.simulate_resume(scheme, dt, K * dt, R, seed, K + 1)
    finally:
        h.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_resume_split_at_benchmark_size(Bd, scheme):
    """100-station DAG, 10,000 replications, full horizon: the run split at
    step 5,000 adds up to the uninterrupted run bit for bit."""
    run = W.layered_dag()
    K = Bd.num_steps(run.dt, run.T)
    h = Bd.EulerNet(run.net)
    try:
        whole = h.simulate(scheme, run.dt, run.T, run.R, run.seed).cpu().numpy()
        cut = K // 2
        s1, N1 = h.simulate_resume(scheme, run.dt, cut * run.dt, run.R, run.seed, 0, state_out=True)
        s2, N2 = h.simulate_resume(scheme, run.dt, run.T, run.R, run.seed, cut, state_in=N1, state_out=True)
        n, R = run.net.n, run.R
        a, b = s1.cpu().numpy(), s2.cpu().numpy()
        head = 5 * n + 4 * R
        assert np.array_equal(a[:head] + b[:head], whole[:head])
        assert np.array_equal(b[head:], whole[head:])
        assert np.array_equal(N2.cpu().numpy().sum(axis=1), whole[head:])
    finally:
        h.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_coupled_gradient_dag100_matches_oracle(Bd, orc, scheme):
    """The 100-station DAG with sinusoid arrivals (64 replications, 200
    steps): two mu_i and two arrival windows, replayed from checkpoints in
    the HBM form's default launch shape."""
    g = W.sinusoid_dag()
    net, dt, T, R, windows, delta = g.net, g.dt, 2.0, 64, 5, 0.05
    params = [0, 57, net.n + 1, net.n + 4]
    h = Bd.EulerNet(net)
    try:
        got = h.grad_coupled(scheme, dt, T, R, 7, windows, delta, params=params)
    finally:
        h.close()
    want = orc.grad_coupled(net, scheme, dt, T, R, 7, windows, delta, params=params)
    assert np.array_equal(got["grad"].cpu().numpy(), want["grad"])
    assert np.allclose(got["var"].cpu().numpy(), want["var"], rtol=1e-9, atol=0.0)
    assert np.all(want["var"] >= 0) and np.any(want["grad"] != 0)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("case", [0, 1])
def test_coupled_gradient_matches_oracle(Bd, orc, scheme, case):
    """Every mu_i and every arrival window, replayed from the device's own
    checkpoints: the mean is bit for bit the oracle's (exact integer sums),
    the variance to 1e-9 relative (sums of squares in another order)."""
    if case == 0:
        net, dt, T, R, windows = _queueing_net(), 0.3, 3.0, 150, 3
    else:
        rng = np.random.default_rng(12)
        net = W.random_small_dag(rng, 5, max_deg=2, m_range=(2, 8), ext_frac=0.7, lam_scale=10.0)
        dt, T, R, windows = 0.05, 2.0, 70, 4
    delta = 0.05
    h = Bd.EulerNet(net)
    try:
        h.set_option(Bd.OPT_HBM_CHUNK, 32)
        g = h.grad_coupled(scheme, dt, T, R, 19, windows, delta, rep_begin=3)
        sub = h.grad_coupled(scheme, dt, T, R, 19, windows, delta, params=[net.n + windows - 1, 0],
                             rep_begin=3)
        # the handle is left as it was: a plain run afterwards is unchanged
        after = h.simulate(scheme, dt, T, R, 19).cpu().numpy()
    finally:
        h.close()
    want = orc.grad_coupled(net, scheme, dt, T, R, 19, windows, delta, rep_begin=3)
    gg, gv = g["grad"].cpu().numpy(), g["var"].cpu().numpy()
    assert np.array_equal(gg, want["grad"])
    assert np.allclose(gv, want["var"], rtol=1e-9, atol=0.0)
    assert np.array_equal(sub["grad"].cpu().numpy(), gg[:, [net.n + windows - 1, 0]])
    assert np.array_equal(after, orc.simulate(net, scheme, dt, T, R, 19)["stats"])
