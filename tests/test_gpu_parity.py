"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results (every statistic, every replication) must agree bit for bit:
the two sides evaluate the same written sampler definitions with the same
IEEE float operations and the same counter-based random streams.  Full-size
runs are checked on sampled replications (the oracle re-runs exactly those
replication indices) and through invariants that hold at any size.
"""
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


def _gpu_stats(Bd, net, scheme, dt, T, R, seed, rep_begin=0, options=None):
    h = Bd.EulerNet(net)
    try:
        for k, v in (options or {}).items():
            h.set_option(k, v)
        return h.simulate(scheme, dt, T, R, seed, rep_begin).cpu().numpy()
    finally:
        h.close()


def _assert_equal(got, want, what):
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{what}: {len(bad)} entries differ, first {bad[:6].tolist()}: "
                             f"gpu {got[bad[:6]].tolist()} oracle {want[bad[:6]].tolist()}")


def _invariants(Bd, stats, net, R):
    sp = Bd.split_stats(stats, net.n, R)
    st, rp, nk = sp["station"], sp["rep"], sp["NK"]
    assert st[:, 0].sum() == rp[:, 0].sum()
    assert st[:, 2].sum() == rp[:, 1].sum()
    assert st[:, 3].sum() == rp[:, 2].sum()
    assert st[:, 4].sum() == rp[:, 3].sum()
    assert (st[:, 1] <= st[:, 0]).all() and (st >= 0).all() and (rp >= 0).all()
    n0 = 0 if net.N0 is None else int(net.N0.sum())
    assert nk.sum() == R * n0 + rp[:, 3].sum() - rp[:, 2].sum()


@pytest.mark.parametrize("scheme", [0, 1])
def test_tandem_full_parity(Bd, orc, scheme):
    """3-station tandem, 1,000 replications x 2,400 steps: every entry."""
    run = W.tandem3()
    got = _gpu_stats(Bd, run.net, scheme, run.dt, run.T, run.R, run.seed)
    want = orc.simulate(run.net, scheme, run.dt, run.T, run.R, run.seed)["stats"]
    _assert_equal(got, want, f"tandem scheme {scheme}")
    _invariants(Bd, got, run.net, run.R)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_dag100_full_size_sampled(Bd, orc, scheme, form):
    """100-station layered DAG at full size (10,000 replications x 10,000
    steps; form 0 = the planner's choice, the benchmark's launch, and the
    persistent form): sampled replications re-run by the oracle must match
    exactly; invariants over all replications."""
    run = W.layered_dag()
    got = _gpu_stats(Bd, run.net, scheme, run.dt, run.T, run.R, run.seed,
                     options={Bd.OPT_FORM: form} if form else None)
    _invariants(Bd, got, run.net, run.R)
    rng = np.random.default_rng(123)
    reps = sorted({0, 1, 31, 32, 5000, run.R - 1} | set(rng.integers(0, run.R, 4).tolist()))
    rp = Bd.split_stats(got, run.net.n, run.R)["rep"]
    for r in reps:
        want = orc.simulate(run.net, scheme, run.dt, run.T, 1, run.seed, rep_begin=r)["rep"][0]
        _assert_equal(rp[r], want, f"dag100 scheme {scheme} replication {r}")


def _small_cases():
    rng = np.random.default_rng(2024)
    cases = []
    for n, R, dt, T in [(1, 1, 0.1, 1.0), (2, 31, 0.07, 2.0), (7, 33, 0.05, 1.23), (33, 100, 0.02, 0.5),
                        (64, 65, 0.1, 3.0), (5, 257, 0.2, 4.1)]:
        net = W.random_small_dag(rng, n, max_deg=3, m_range=(1, 12), ext_frac=0.6, lam_scale=30.0)
        if n > 2:
            net.N0 = rng.integers(0, 15, size=n).astype(np.int32)
        cases.append((net, R, dt, T))
    # table arrivals, a row without exit, large means (PTRS / BTRS paths)
    row_ptr, col, prob = W.csr_from_edges(4, [(0, 1, 0.25), (0, 2, 0.75), (1, 3, 1.0), (2, 3, 0.5)])
    tab = np.array([[300.0, 0, 0, 0], [2000.0, 0, 0, 40.0], [50.0, 0, 0, 5.0]])
    net = W.Network(4, row_ptr, col, prob, np.array([400, 5, 900, 30]), np.array([2.0, 9.0, 0.7, 1.5]),
                    W.Arrivals(kind=W.ARR_TABLE, table=tab, tab_dt=0.4))
    cases.append((net, 70, 0.05, 1.5))
    return cases


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("scheme", [0, 1])
def test_small_networks_parity(Bd, orc, case, scheme):
    """Random DAGs with skip edges, ragged R and T/dt, initial customers,
    table arrivals and heavy-traffic stations: every entry."""
    net, R, dt, T = _small_cases()[case]
    got = _gpu_stats(Bd, net, scheme, dt, T, R, 1000 + case)
    want = orc.simulate(net, scheme, dt, T, R, 1000 + case)["stats"]
    _assert_equal(got, want, f"case {case} scheme {scheme}")


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("scheme", [0, 1])
def test_small_networks_hbm_form_parity(Bd, orc, case, scheme):
    """The HBM form on the same cases: skip edges across several levels make
    the skewed forward scheme keep routed counts for more than one step
    (ring depth > 2); one and five steps per graph replay; replications run
    in chunks of 32 (several chunks and a ragged one)."""
    net, R, dt, T = _small_cases()[case]
    want = orc.simulate(net, scheme, dt, T, R, 1000 + case)["stats"]
    for steps, chunk in ((1, 0), (5, 0), (5, 32)):
        got = _gpu_stats(Bd, net, scheme, dt, T, R, 1000 + case,
                         options={Bd.OPT_FORM: 2, Bd.OPT_GRAPH_STEPS: steps, Bd.OPT_HBM_CHUNK: chunk})
        _assert_equal(got, want, f"hbm case {case} scheme {scheme} graph steps {steps} chunk {chunk}")


@pytest.mark.parametrize("scheme", [0, 1])
def test_launch_shape_and_form_invariance(Bd, scheme):
    """Counter-based keying: tile size, block, grid and the HBM/graph form do
    not change any result."""
    rng = np.random.default_rng(9)
    net = W.random_small_dag(rng, 24, max_deg=3, m_range=(2, 20), ext_frac=0.5, lam_scale=20.0)
    R, dt, T, seed = 200, 0.05, 2.0, 77
    ref = _gpu_stats(Bd, net, scheme, dt, T, R, seed)
    variants = [{Bd.OPT_FORM: 1, Bd.OPT_TILE_REPS: 1, Bd.OPT_BLOCK: 64}, {Bd.OPT_FORM: 1, Bd.OPT_TILE_REPS: 8},
                {Bd.OPT_FORM: 1, Bd.OPT_TILE_REPS: 32, Bd.OPT_GRID: 1},
                {Bd.OPT_FORM: 1, Bd.OPT_TILE_REPS: 64, Bd.OPT_BLOCK: 128},
                {Bd.OPT_FORM: 2}, {Bd.OPT_FORM: 2, Bd.OPT_GRAPH_STEPS: 7, Bd.OPT_BLOCK: 64},
                {Bd.OPT_FORM: 3, Bd.OPT_PIPE_WARPS: 1}, {Bd.OPT_FORM: 3, Bd.OPT_PIPE_WARPS: 5},
                {Bd.OPT_FORM: 3, Bd.OPT_PIPE_WARPS: 16, Bd.OPT_GRID: 3}]
    for opt in variants:
        _assert_equal(_gpu_stats(Bd, net, scheme, dt, T, R, seed, options=opt), ref, f"options {opt}")


def test_rep_begin_split(Bd):
    """A replication range split over two calls gives the same results."""
    run = W.tandem3(R=300)
    full = _gpu_stats(Bd, run.net, 1, run.dt, 5.0, 300, 5)
    a = _gpu_stats(Bd, run.net, 1, run.dt, 5.0, 120, 5, rep_begin=0)
    b = _gpu_stats(Bd, run.net, 1, run.dt, 5.0, 180, 5, rep_begin=120)
    n = run.net.n
    sf, sa, sb = (Bd.split_stats(x, n, r) for x, r in ((full, 300), (a, 120), (b, 180)))
    _assert_equal(sf["rep"].ravel(), np.concatenate([sa["rep"], sb["rep"]]).ravel(), "rep split")
    _assert_equal(sf["station"].ravel(), (sa["station"] + sb["station"]).ravel(), "station split")


@pytest.mark.parametrize("scheme", [0, 1])
def test_hbm_form_parity(Bd, orc, scheme):
    """The per-step HBM-state kernels under a CUDA graph match the oracle."""
    run = W.tandem3(R=77)
    got = _gpu_stats(Bd, run.net, scheme, run.dt, 3.0, run.R, 3, options={Bd.OPT_FORM: 2})
    want = orc.simulate(run.net, scheme, run.dt, 3.0, run.R, 3)["stats"]
    _assert_equal(got, want, "hbm form")


@pytest.mark.parametrize("s", [10, 100])
@pytest.mark.parametrize("scheme", [0, 1])
def test_scale_dag_full_size_sampled(Bd, orc, s, scheme):
    """The scale sweep's 2,000-station DAG at its full size, 100,000
    replications over the full horizon (s = 10: K = 159; s = 100: K = 500):
    sampled replications re-run by the oracle, invariants over all."""
    run = W.scale_dag(s)
    got = _gpu_stats(Bd, run.net, scheme, run.dt, run.T, run.R, run.seed)
    _invariants(Bd, got, run.net, run.R)
    rp = Bd.split_stats(got, run.net.n, run.R)["rep"]
    for r in (0, 54321, run.R - 1):
        want = orc.simulate(run.net, scheme, run.dt, run.T, 1, run.seed, rep_begin=r)["rep"][0]
        _assert_equal(rp[r], want, f"scale {s} replication {r}")


@pytest.mark.parametrize("s", [10, 10000])
def test_scale_dag_sampled(Bd, orc, s):
    """2,000-station DAG of the scale sweep: GPU run over 2,048 replications,
    sampled replications re-run by the oracle."""
    run = W.scale_dag(s, R=2048)
    T = run.T if s == 10 else 5.0
    got = _gpu_stats(Bd, run.net, 1, run.dt, T, run.R, run.seed)
    _invariants(Bd, got, run.net, run.R)
    rp = Bd.split_stats(got, run.net.n, run.R)["rep"]
    for r in (0, 777, run.R - 1):
        want = orc.simulate(run.net, 1, run.dt, T, 1, run.seed, rep_begin=r)["rep"][0]
        _assert_equal(rp[r], want, f"scale {s} replication {r}")


def test_simulate_host_matches_device(Bd):
    run = W.tandem3(R=50)
    h = Bd.EulerNet(run.net)
    try:
        dev = h.simulate(0, run.dt, 2.0, 50, 8).cpu().numpy()
        host = h.simulate_host(0, run.dt, 2.0, 50, 8)
    finally:
        h.close()
    _assert_equal(host, dev, "host entry point")


def test_zero_replications(Bd):
    import torch
    run = W.tandem3(R=1)
    h = Bd.EulerNet(run.net)
    try:
        out = torch.full((Bd.stats_len(3, 0),), 7, dtype=torch.int64, device="cuda")
        h.simulate(0, run.dt, 1.0, 0, 1, stats=out)
        assert (out == 0).all()
    finally:
        h.close()


def test_sampler_cap_reports_error(Bd):
    """A rejection loop that hits its (lowered) cap returns an error status;
    nothing faults or hangs."""
    run = W.single_station(1000, 1.0, 3000.0, 0.01, 1.0, 64, 1)
    h = Bd.EulerNet(run.net)
    try:
        h.set_option(Bd.OPT_SAMPLER_CAP, 1)
        with pytest.raises(Bd.EulerError) as ei:
            h.simulate(0, 0.01, 1.0, 64, 1)
        assert ei.value.code == -5
        h.set_option(Bd.OPT_SAMPLER_CAP, -1)
        h.simulate(0, 0.01, 1.0, 64, 1)  # status was cleared; default cap works
    finally:
        h.close()


def test_pipeline_wait_timeout_reports_error(Bd):
    """A bounded inter-warp wait that runs out (the warps withhold their
    progress on purpose) ends the kernel with EULER_ERR_STALL; the context stays usable."""
    rng = np.random.default_rng(4)
    net = W.random_small_dag(rng, 12, max_deg=2, m_range=(2, 9), ext_frac=0.8, lam_scale=5.0)
    h = Bd.EulerNet(net)
    try:
        h.set_option(Bd.OPT_FORM, 3)
        h.set_option(Bd.OPT_PIPE_WARPS, 4)
        h.set_option(Bd.OPT_WAIT_LIMIT, 20000)  # roughly a few milliseconds per wait
        h.set_option(Bd.OPT_TEST_STALL, 1)
        with pytest.raises(Bd.EulerError) as ei:
            h.simulate(1, 0.1, 2.0, 64, 3)
        assert ei.value.code == -8
        h.set_option(Bd.OPT_TEST_STALL, -1)
        h.set_option(Bd.OPT_WAIT_LIMIT, -1)
        ok = h.simulate(1, 0.1, 2.0, 64, 3).cpu().numpy()  # usable afterwards
        assert ok[: 5 * 12].sum() > 0
    finally:
        h.close()


def test_overflow_reports_error(Bd, orc):
    """A station whose count passes 2^30 latches EULER_ERR_OVERFLOW."""
    run = W.single_station(1, 1e-6, 1e6, 1.0, 1100.0, 32, 1)
    h = Bd.EulerNet(run.net)
    try:
        with pytest.raises(Bd.EulerError) as ei:
            h.simulate(0, 1.0, 1100.0, 32, 1)
        assert ei.value.code == -6
    finally:
        h.close()
    assert orc.simulate(run.net, 0, 1.0, 1100.0, 32, 1, expect_ok=False)["rc"] == -6
