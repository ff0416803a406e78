"""GPU parity of the widening rows: the average scheme and the step-size
rule, the Eq. (1)/(2) departure samplers, and time-varying staffing."""
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


def _net(seed=21, n=14):
    rng = np.random.default_rng(seed)
    net = W.random_small_dag(rng, n, max_deg=3, m_range=(1, 12), ext_frac=0.6, lam_scale=25.0)
    net.N0 = rng.integers(0, 10, size=n).astype(np.int32)
    return net


def test_average_scheme(Bd, orc):
    net = _net()
    h = Bd.EulerNet(net)
    try:
        avg, sb, sf = h.simulate_average(0.05, 1.7, 90, 12, rep_begin=3)
        dt = h.select_dt()
        dt2 = h.select_dt(0.2)
    finally:
        h.close()
    ob = orc.simulate(net, 0, 0.05, 1.7, 90, 12, rep_begin=3)["stats"]
    of = orc.simulate(net, 1, 0.05, 1.7, 90, 12, rep_begin=3)["stats"]
    assert np.array_equal(sb.cpu().numpy(), ob) and np.array_equal(sf.cpu().numpy(), of)
    assert np.array_equal(avg.cpu().numpy(), 0.5 * (ob.astype(np.float64) + of))
    assert math.isclose(dt, 0.4 / math.sqrt(net.servers.max()) / net.mu.max(), rel_tol=1e-15)
    assert math.isclose(dt2, 0.2 / net.mu.max(), rel_tol=1e-15)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1])
def test_naive_departure_modes(Bd, orc, mode, scheme):
    net = _net(22)
    h = Bd.EulerNet(net)
    try:
        h.set_option(Bd.OPT_DEPARTURE, mode)
        got = h.simulate(scheme, 0.05, 2.0, 77, 3).cpu().numpy()
        with pytest.raises(Bd.EulerError):
            h.grad(scheme, 0.05, 2.0, 8, 3)
    finally:
        h.close()
    old = orc.set_departure_mode(mode)
    try:
        want = orc.simulate(net, scheme, 0.05, 2.0, 77, 3)["stats"]
    finally:
        orc.set_departure_mode(old)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("scheme", [0, 1])
def test_staffing_schedule(Bd, orc, scheme):
    net = _net(23)
    rng = np.random.default_rng(5)
    net.servers_schedule = rng.integers(1, 15, size=(5, net.n)).astype(np.int32)
    net.servers_schedule_dt = 0.4
    h = Bd.EulerNet(net)
    try:
        got = h.simulate(scheme, 0.05, 2.5, 70, 4).cpu().numpy()
        g = h.grad(scheme, 0.05, 2.5, 40, 4, scores=True)
    finally:
        h.close()
    want = orc.simulate(net, scheme, 0.05, 2.5, 70, 4)["stats"]
    assert np.array_equal(got, want)
    og = orc.grad(net, scheme, 0.05, 2.5, 40, 4, scores=True)
    assert np.array_equal(g["scores"].cpu().numpy(), og["scores"])
