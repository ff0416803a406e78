"""Host-side checks of the roofline's operation model and of the synthetic
workload generators (CPU, no GPU).

The operation model prices every work counter of the oracle, so that the
algorithmic operations per unit follow the events the oracle actually counts.
The 100-station generator implements the configuration's staffing: layer-0
stations at utilisation 0.9, every downstream station restaffed from the
traffic equations (Sec. 3.3) to a utilisation of at most 0.9.
"""
import numpy as np

from oracle import oracle as O
from paper_2402_13259_gb300 import opmodel
from paper_2402_13259_gb300 import workloads as W


def test_every_counter_is_priced():
    assert set(opmodel.COST) == set(O.COUNTER_NAMES)
    assert all(v > 0 for v in opmodel.COST.values())


def test_ops_per_unit_follow_the_counted_events(orc):
    run = W.layered_dag()
    orc.counters_reset()
    orc.simulate(run.net, orc.BACKWARD, run.dt, 2.0, 2, run.seed)
    c = orc.counters()
    ops = opmodel.ops_per_unit(c)
    # a unit is at least its bookkeeping, one Philox block's share and one draw
    floor = opmodel.COST["units"] + opmodel.COST["uniforms"]
    assert ops > floor
    # doubling every count but the units doubles the per-unit cost of the events
    c2 = {k: (v if k == "units" else 2 * v) for k, v in c.items()}
    assert abs(opmodel.ops_per_unit(c2) - (2 * ops - opmodel.COST["units"])) < 1e-6 * ops


def _traffic(net):
    """Total arrival rates lambda~ = lambda + P^T lambda~ (stations numbered in
    flow order), from the network's per-station external rates."""
    lam = net.arrivals.w * net.arrivals.a if net.arrivals.kind == W.ARR_SINUSOID else net.arrivals.w
    tot = np.array(lam, dtype=float)
    for i in range(net.n):
        for e in range(int(net.row_ptr[i]), int(net.row_ptr[i + 1])):
            tot[int(net.col[e])] += net.prob[e] * tot[i]
    return tot


def test_dag100_staffing_keeps_every_utilisation_at_most_0_9():
    net = W.layered_dag().net
    tot = _traffic(net)
    rho = tot / (net.servers * net.mu)
    reached = tot > 0
    assert reached.all()  # every station receives customers
    assert (rho[reached] <= 0.9 + 1e-9).all()
    ext = net.arrivals.w > 0
    assert np.allclose(rho[ext], 0.9, rtol=1e-6)  # layer 0 at 0.9 exactly
    assert (net.servers >= 1).all() and (net.mu >= 0.5 - 1e-12).all() and (net.mu <= 2.0 + 1e-12).all()
