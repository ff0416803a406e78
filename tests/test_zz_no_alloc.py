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


def test_noalloc_rejects_runs_beyond_its_scratch(Bd):
    run = W.tandem3(R=1)
    h = Bd.EulerNet(run.net)
    try:
        with pytest.raises(Bd.EulerError) as ei:
            _noalloc(Bd, h, 0, run.dt, 1.0, 3_000_000, 1)
        assert ei.value.code == -7 and "64 MiB" in str(ei.value)
    finally:
        h.close()
