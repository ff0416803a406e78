"""GPU parity of the sojourn-time sampler (Sec. 6, Algorithm 4).

The kernel advances the tagged customers while the Euler time loop runs; the
oracle stores the whole sample paths and runs Algorithm 4 over them.  Every
sojourn (in steps, censored ones negative) and the paths' statistics must
agree bit for bit.
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


def _gpu(Bd, net, scheme, dt, T, R, seed, station, tau0, samples, rep_begin=0, options=None):
    import torch
    h = Bd.EulerNet(net)
    try:
        for k, v in (options or {}).items():
            h.set_option(k, v)
        stats = torch.empty(Bd.stats_len(net.n, R), dtype=torch.int64, device="cuda")
        out = h.sojourn(scheme, dt, T, R, seed, station, tau0, samples, rep_begin, stats=stats)
        plain = h.simulate(scheme, dt, T, R, seed, rep_begin).cpu().numpy()
        return out.cpu().numpy(), stats.cpu().numpy(), plain
    finally:
        h.close()


def _assert_equal(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} entries differ, first {bad[:4].tolist()}: "
                             f"gpu {[got[tuple(b)] for b in bad[:4]]} "
                             f"oracle {[want[tuple(b)] for b in bad[:4]]}")


def _check(Bd, orc, net, scheme, dt, T, R, seed, station, tau0, samples, rep_begin=0, options=None):
    got, st, plain = _gpu(Bd, net, scheme, dt, T, R, seed, station, tau0, samples, rep_begin, options)
    want = orc.sojourn(net, scheme, dt, T, R, seed, station, tau0, samples, rep_begin)
    _assert_equal(got, want["steps"], f"sojourn scheme {scheme}")
    _assert_equal(st, want["stats"], f"sojourn stats scheme {scheme}")
    _assert_equal(st, plain, f"sojourn vs simulate stats scheme {scheme}")
    return got


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
def test_tandem_sojourn_parity(Bd, orc, scheme, form):
    """3-station tandem, 200 replications (6 full tiles and a ragged one), 3
    tagged customers each, entering mid-run; the persistent form (customers in
    shared memory) and the HBM form (customers in global memory)."""
    run = W.tandem3()
    got = _check(Bd, orc, run.net, scheme, run.dt, 6.0, 200, run.seed, 0, 100, 3,
                 options={Bd.OPT_FORM: form})
    assert (got > 0).mean() > 0.5


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("seed", [3, 8])
def test_random_dag_sojourn_parity(Bd, orc, scheme, seed, form):
    """Random small DAGs (skips across layers, several out-edges, queues that
    build and drain), several entry stations and steps, a replication offset;
    both forms."""
    rng = np.random.default_rng(seed)
    net = W.random_small_dag(rng, 9, max_deg=3, m_range=(1, 6), ext_frac=0.5, lam_scale=6.0)
    net.N0 = rng.integers(0, 12, size=net.n).astype(np.int32)
    for station, tau0 in [(0, 1), (int(rng.integers(0, net.n)), 37), (net.n - 1, 150)]:
        _check(Bd, orc, net, scheme, 0.05, 12.0, 75, 11 + seed, station, tau0, 2, rep_begin=7,
               options={Bd.OPT_FORM: form, Bd.OPT_HBM_CHUNK: 32 if seed == 8 else 0})


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
def test_dag100_sojourn_parity(Bd, orc, scheme, form):
    """The 100-station layered DAG, 70 replications x 300 steps, both forms."""
    run = W.layered_dag()
    _check(Bd, orc, run.net, scheme, run.dt, 3.0, 70, run.seed, 3, 20, 2, options={Bd.OPT_FORM: form})


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_with_staffing_and_departure_variants(Bd, orc, scheme, form):
    """The staffing-schedule and Eq. (1)/(2) instantiations of the kernels."""
    rng = np.random.default_rng(21)
    net = W.random_small_dag(rng, 7, max_deg=2, m_range=(1, 8), ext_frac=0.6, lam_scale=5.0)
    net.servers_schedule = rng.integers(1, 9, size=(4, net.n)).astype(np.int32)
    net.servers_schedule_dt = 1.5
    _check(Bd, orc, net, scheme, 0.05, 8.0, 64, 5, 0, 10, 2, options={Bd.OPT_FORM: form})
    net.servers_schedule = None
    for mode in (1, 2):
        old = orc.set_departure_mode(mode)
        try:
            _check(Bd, orc, net, scheme, 0.05, 8.0, 40, 6, 0, 10, 2,
                   options={Bd.OPT_DEPARTURE: mode, Bd.OPT_FORM: form})
        finally:
            orc.set_departure_mode(old)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
def test_sojourn_edge_cases(Bd, orc, scheme, form):
    """Entry in the last step (all censored, nothing accounted), entry in the
    first step, many tagged customers (the persistent tile shrinks below 32
    replications), and no replications at all."""
    import torch
    run = W.tandem3()
    K = Bd.num_steps(run.dt, 2.0)
    o = {Bd.OPT_FORM: form}
    got = _check(Bd, orc, run.net, scheme, run.dt, 2.0, 40, 4, 1, K, 3, options=o)
    assert (got == 0).all()
    _check(Bd, orc, run.net, scheme, run.dt, 2.0, 40, 4, 0, 1, 1, options=o)
    _check(Bd, orc, run.net, scheme, run.dt, 1.0, 37, 4, 0, 30, 700, options=o)
    h = Bd.EulerNet(run.net)
    try:
        out = torch.empty((0, 2), dtype=torch.int32, device="cuda")
        h.sojourn(scheme, run.dt, 1.0, 0, 4, 0, 5, 2, out=out)
        for bad in [dict(station=3, tau0=5), dict(station=0, tau0=0), dict(station=0, tau0=K + 1)]:
            with pytest.raises(Bd.EulerError):
                h.sojourn(scheme, run.dt, 2.0, 4, 4, samples=1, **bad)
    finally:
        h.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_dag100_full_size_sojourn_sampled(Bd, orc, scheme):
    """The benchmark workload at full size (10,000 replications x 10,000
    steps; the planner's form) with 4 tagged customers per replication
    entering station 0 at t = 50: sampled replications re-run by the oracle
    match exactly; the statistics equal those of the plain simulation."""
    import torch
    run = W.layered_dag()
    h = Bd.EulerNet(run.net)
    try:
        stats = torch.empty(Bd.stats_len(run.net.n, run.R), dtype=torch.int64, device="cuda")
        out = h.sojourn(scheme, run.dt, run.T, run.R, run.seed, 0, 5000, 4, stats=stats).cpu().numpy()
        plain = h.simulate(scheme, run.dt, run.T, run.R, run.seed).cpu().numpy()
    finally:
        h.close()
    _assert_equal(stats.cpu().numpy(), plain, "full-size sojourn stats")
    assert (out > 0).mean() > 0.9
    for r in (0, 33, run.R - 1):
        want = orc.sojourn(run.net, scheme, run.dt, run.T, 1, run.seed, 0, 5000, 4, rep_begin=r)
        _assert_equal(out[r:r + 1], want["steps"], f"full-size replication {r}")
