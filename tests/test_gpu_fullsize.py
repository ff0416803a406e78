"""Full-size parity on the benchmark configurations, in the launch form the
benchmark times: the scale sweep's 2,000-station DAG at s = 1000 and
s = 10,000 over the whole horizon with all 100,000 replications, and the
100-station DAG's step-level state N_tau (Sec. 2.2) at two cuts of the full
run.  Sampled replications are re-run by the oracle (counter-based keying
makes a replication's trajectory independent of the others); the oracle works
while the GPU runs.
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


def _equal(got, want, what):
    got, want = np.asarray(got), np.asarray(want)
    if not np.array_equal(got, want):
        bad = np.nonzero(got.ravel() != want.ravel())[0]
        raise AssertionError(f"{what}: {len(bad)} entries differ, first {bad[:6].tolist()}: "
                             f"gpu {got.ravel()[bad[:6]].tolist()} oracle {want.ravel()[bad[:6]].tolist()}")


def _invariants(Bd, stats, net, R):
    sp = Bd.split_stats(stats, net.n, R)
    st, rp, nk = sp["station"], sp["rep"], sp["NK"]
    assert st[:, 0].sum() == rp[:, 0].sum()
    assert st[:, 2].sum() == rp[:, 1].sum()
    assert st[:, 3].sum() == rp[:, 2].sum()
    assert st[:, 4].sum() == rp[:, 3].sum()
    assert (st[:, 1] <= st[:, 0]).all() and (st >= 0).all() and (rp >= 0).all()
    assert nk.sum() == rp[:, 3].sum() - rp[:, 2].sum()


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("s", [1000, 10000])
def test_scale_dag_full_horizon(Bd, orc, s, scheme):
    """2,000-station DAG, Halfin-Whitt staffing at scale s, dt = 1/sqrt(s),
    T = 50 (s = 1000: K = 1,582; s = 10,000: K = 5,000), 100,000
    replications in the planner's chunked HBM form: the regime where the
    PTRS and BTRS rejection samplers carry most draws (Sec. 5.3, Theorem 3).
    Three sampled replications match the oracle exactly; invariants hold over
    all."""
    run = W.scale_dag(s)
    h = Bd.EulerNet(run.net)
    try:
        got = h.simulate(scheme, run.dt, run.T, run.R, run.seed, check=False)
        reps = (0, 54321, run.R - 1)
        want = {r: orc.simulate(run.net, scheme, run.dt, run.T, 1, run.seed, rep_begin=r)["rep"][0]
                for r in reps}
        h.status()
        got = got.cpu().numpy()
    finally:
        h.close()
    _invariants(Bd, got, run.net, run.R)
    rp = Bd.split_stats(got, run.net.n, run.R)["rep"]
    for r in reps:
        _equal(rp[r], want[r], f"scale {s} scheme {scheme} replication {r}")


@pytest.mark.parametrize("scheme", [0, 1])
def test_dag100_state_at_cuts(Bd, orc, scheme):
    """100-station DAG at full size (10,000 replications, K = 10,000), run in
    three parts through the checkpoint entry point: N_tau of every station at
    the cuts tau = 2,500 and 7,500 equals the oracle's trajectory for the
    sampled replications, and so does each part's per-replication
    statistics; the parts add up to the uninterrupted run."""
    run = W.layered_dag()
    n, R = run.net.n, run.R
    K = Bd.num_steps(run.dt, run.T)
    cuts = (0, 2500, 7500, K)
    reps = (0, 31, 4097, R - 1)
    h = Bd.EulerNet(run.net)
    try:
        whole = h.simulate(scheme, run.dt, run.T, R, run.seed, check=False)
        parts, states = [], []
        Nd = None
        for a, b in zip(cuts[:-1], cuts[1:]):
            st, Nd = h.simulate_resume(scheme, run.dt, b * run.dt, R, run.seed, a, state_in=Nd,
                                       state_out=True, check=False)
            parts.append(st)
            states.append(Nd)
        # the oracle's trajectories of the sampled replications to the last cut
        traj = {r: orc.simulate(run.net, scheme, run.dt, cuts[2] * run.dt, 1, run.seed, rep_begin=r,
                                trace=True)["N"][:, :, 0] for r in reps}
        seg = {}
        for r in reps:
            N_in = None
            for k, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
                o = orc.simulate_resume(run.net, scheme, run.dt, b * run.dt, 1, run.seed, a, N_in, rep_begin=r)
                seg[(r, k)] = o
                N_in = o["N_out"]
        h.status()
        whole = whole.cpu().numpy()
        parts = [p.cpu().numpy() for p in parts]
        states = [s_.cpu().numpy() for s_ in states]
    finally:
        h.close()
    head = 5 * n + 4 * R
    _equal(sum(p[:head] for p in parts), whole[:head], "parts add up")
    _equal(parts[-1][head:], whole[head:], "N_K")
    for r in reps:
        for k, cut in ((0, cuts[1]), (1, cuts[2])):
            _equal(states[k][:, r], traj[r][cut - 1], f"scheme {scheme} N at step {cut}, replication {r}")
        for k in range(3):
            rp = Bd.split_stats(parts[k], n, R)["rep"][r]
            _equal(rp, seg[(r, k)]["rep"][0], f"scheme {scheme} part {k} replication {r}")
            _equal(states[k][:, r], seg[(r, k)]["N_out"][:, 0], f"scheme {scheme} part {k} N_out replication {r}")
