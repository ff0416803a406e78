"""euler_net_simulate_noalloc: the entry point for callers that cannot
allocate device memory while they run (fixed device-memory budgets, plug-ins
whose host owns the allocator, loops where a cudaMalloc/cudaFree and the
synchronisation it may bring are not acceptable).  It must give exactly the
results of euler_net_simulate, call after call, although every call reuses
the same reserved scratch area.

Collected last on purpose (file name), so a failure here comes after every
other test has run.
"""
import ctypes as C

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


def _noalloc(Bd, h, scheme, dt, T, R, seed, rep_begin=0):
    import torch
    out = torch.full((Bd.stats_len(h.n, R),), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = Bd.lib().euler_net_simulate_noalloc(h._h, scheme, dt, T, R, seed, rep_begin,
                                             C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    if rc != 0:
        raise Bd.EulerError(rc, Bd.lib().euler_net_last_error().decode())
    h.status()
    return out.cpu().numpy()


@pytest.mark.parametrize("scheme", [0, 1])
def test_noalloc_matches_simulate_on_consecutive_calls(Bd, scheme):
    rng = np.random.default_rng(31)
    net = W.random_small_dag(rng, 12, max_deg=3, m_range=(1, 15), ext_frac=0.6, lam_scale=25.0)
    net.N0 = rng.integers(0, 9, size=12).astype(np.int32)
    h = Bd.EulerNet(net)
    try:
        # two calls in a row on the shared scratch: a larger run, then a smaller
        # one with another seed and replication offset (stale contents must not leak)
        for R, seed, rep_begin, T in ((150, 5, 0, 1.7), (70, 6, 33, 1.1)):
            want = h.simulate(scheme, 0.05, T, R, seed, rep_begin).cpu().numpy()
            got = _noalloc(Bd, h, scheme, 0.05, T, R, seed, rep_begin)
            assert np.array_equal(got, want), np.nonzero(got != want)[0][:8]
    finally:
        h.close()


def _chunk_cases():
    """Networks whose per-step tables take several staging chunks: more than
    819 stations (departure constants), K x n_ex > 4096 (arrival means), a
    staffing schedule over more rows than one chunk holds and one with rows
    longer than a chunk (n > 4096), and the Eq. (1)/(2) departure samplers."""
    rng = np.random.default_rng(77)
    cases = []
    big = W.random_small_dag(rng, 1100, max_deg=2, m_range=(1, 6), ext_frac=0.1, lam_scale=4.0)
    cases.append(("stations>819", big, 40, 0.1, 1.0, None, 0))
    ext = W.random_small_dag(rng, 12, max_deg=3, m_range=(1, 15), ext_frac=0.6, lam_scale=25.0)
    cases.append(("K*n_ex>4096", ext, 36, 0.01, 7.3, None, 0))
    sched = np.maximum(1, rng.integers(1, 15, size=(5, 12))).astype(np.int32)
    cases.append(("schedule", ext, 36, 0.01, 7.3, (sched, 1.7), 0))
    wide = W.random_small_dag(rng, 4100, max_deg=1, m_range=(1, 4), ext_frac=0.05, lam_scale=3.0)
    wsched = rng.integers(1, 5, size=(3, 4100)).astype(np.int32)
    cases.append(("schedule rows>4096", wide, 33, 0.1, 2.0, (wsched, 0.7), 0))
    cases.append(("Eq. (1)", ext, 36, 0.05, 2.0, None, 1))
    cases.append(("Eq. (2)", ext, 36, 0.05, 2.0, None, 2))
    return cases


@pytest.mark.parametrize("case", range(6))
@pytest.mark.parametrize("scheme", [0, 1])
def test_noalloc_staging_chunks(Bd, scheme, case):
    """Tables staged over several chunks give euler_net_simulate's results;
    a repeated call reuses the tables held in the scratch and still agrees."""
    name, net, R, dt, T, sched, dep = _chunk_cases()[case]
    h = Bd.EulerNet(net)
    try:
        if sched is not None:
            h.set_servers_schedule(*sched)
        if dep:
            h.set_option(Bd.OPT_DEPARTURE, dep)
        want = h.simulate(scheme, dt, T, R, 3, 5).cpu().numpy()
        for _ in range(2):
            got = _noalloc(Bd, h, scheme, dt, T, R, 3, 5)
            assert np.array_equal(got, want), (name, np.nonzero(got != want)[0][:8])
    finally:
        h.close()


def test_noalloc_tables_follow_handle_changes(Bd):
    """A staffing schedule set (or cleared) between two calls with the same
    (dt, T) is seen by the second call, and a second handle's call does not
    reuse the first handle's tables."""
    rng = np.random.default_rng(5)
    net = W.random_small_dag(rng, 10, max_deg=2, m_range=(2, 9), ext_frac=0.5, lam_scale=12.0)
    other = W.random_small_dag(rng, 10, max_deg=2, m_range=(2, 9), ext_frac=0.5, lam_scale=30.0)
    h, g = Bd.EulerNet(net), Bd.EulerNet(other)
    try:
        dt, T, R = 0.05, 2.0, 40
        a = _noalloc(Bd, h, 1, dt, T, R, 9)
        assert np.array_equal(a, h.simulate(1, dt, T, R, 9).cpu().numpy())
        h.set_servers_schedule(np.full((2, 10), 1, dtype=np.int32), 1.0)
        b = _noalloc(Bd, h, 1, dt, T, R, 9)
        assert np.array_equal(b, h.simulate(1, dt, T, R, 9).cpu().numpy()) and not np.array_equal(a, b)
        c = _noalloc(Bd, g, 1, dt, T, R, 9)
        assert np.array_equal(c, g.simulate(1, dt, T, R, 9).cpu().numpy())
        h.set_servers_schedule(None, 1.0)
        assert np.array_equal(_noalloc(Bd, h, 1, dt, T, R, 9), a)
    finally:
        h.close()
        g.close()


def test_noalloc_rejects_runs_beyond_its_scratch(Bd):
    run = W.tandem3(R=1)
    h = Bd.EulerNet(run.net)
    try:
        with pytest.raises(Bd.EulerError) as ei:
            _noalloc(Bd, h, 0, run.dt, 1.0, 3_000_000, 1)
        assert ei.value.code == -7 and "64 MiB" in str(ei.value)
    finally:
        h.close()
