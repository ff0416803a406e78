"""The batched form: many networks of uneven size and horizon in one
persistent launch must give, for every run, exactly the statistics of that
run launched on its own (and of the CPU oracle)."""
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


def _mixed_batch():
    rng = np.random.default_rng(77)
    nets, runs = [], []
    for k, n in enumerate([1, 3, 6, 17, 40, 90]):
        net = W.random_small_dag(rng, n, max_deg=3, m_range=(1, 25), ext_frac=0.6, lam_scale=20.0)
        nets.append(net)
        runs.append((k % 2, float(rng.choice([0.02, 0.05, 0.1])), float(rng.uniform(0.3, 2.5)),
                     int(rng.integers(1, 150)), 500 + k, int(rng.integers(0, 50))))
    t = W.tandem3()
    nets.append(t.net)
    runs.append((1, t.dt, 3.0, 333, 7, 0))
    d = W.layered_dag()
    nets.append(d.net)
    runs.append((0, d.dt, 2.0, 64, 2, 1000))
    # a 1,500-station DAG: its per-station sums go to the global scratch slot
    big = W.layered_dag(L=15, W=100, seed=11, R=40, T=0.3, dt=0.01).net
    nets.append(big)
    runs.append((1, 0.01, 0.3, 40, 9, 0))
    # networks with n R >= 2^18 units per step: HBM-form items (per-step
    # kernels), one of them twice with another scheme and replication range
    wide = W.layered_dag(R=2800, T=0.3).net
    nets += [wide, wide]
    runs += [(1, 0.01, 0.3, 2800, 3, 17), (0, 0.01, 0.3, 2700, 3, 5000)]
    sc = W.scale_dag(10, R=200)
    nets.append(sc.net)
    runs.append((0, sc.dt, 3.0, 200, 4, 0))
    return nets, runs


def test_batch_matches_single_runs_and_oracle(Bd, orc):
    """Small networks share the persistent launch, large ones (n R >= 2^18)
    run as HBM-form items; before and after autotuning (which may move the
    threshold between the two) every run equals its own launch."""
    nets, runs = _mixed_batch()
    handles = []
    for net in nets:  # a network listed twice shares one handle
        same = [k for k in range(len(handles)) if nets[k] is net]
        handles.append(handles[same[0]] if same else Bd.EulerNet(net))
    try:
        single = []
        for h, r in zip(handles, runs):
            single.append(h.simulate(r[0], r[1], r[2], r[3], r[4], r[5]).cpu().numpy())
        b = Bd.Batch(handles, runs)
        try:
            out = [s.cpu().numpy() for s in b.run()]
            for j, (x, y) in enumerate(zip(out, single)):
                assert np.array_equal(x, y), f"run {j} differs from its single launch"
            assert b.info()["hbm_networks"] == 3  # the three with n R >= 2^18
            blk = b.autotune()
            assert blk in (128, 256, 512)
            info = b.info()
            assert info["block"] == blk and info["hbm_block"] in (128, 256) and info["graph_steps"] in (16, 32, 64)
            assert 0 <= info["hbm_networks"] <= len(runs) and info["tile_shift"] in (-1, 0, 1)
            stats = b.alloc_stats()
            for _ in range(2):  # graph replay on the same buffers
                b.run(stats)
                for j, (x, y) in enumerate(zip(stats, single)):
                    assert np.array_equal(x.cpu().numpy(), y), f"run {j} after autotune"
        finally:
            b.close()
        for j in (0, 1, 2, 3, 6):
            net, r = nets[j], runs[j]
            want = orc.simulate(net, r[0], r[1], r[2], r[3], r[4], rep_begin=r[5])["stats"]
            assert np.array_equal(single[j], want), f"run {j} vs oracle"
        for j in (9, 11):  # HBM-form items: sampled replications against the oracle
            net, r = nets[j], runs[j]
            rp = Bd.split_stats(single[j], net.n, r[3])["rep"]
            for k in (0, r[3] - 1):
                want = orc.simulate(net, r[0], r[1], r[2], 1, r[4], rep_begin=r[5] + k)["rep"][0]
                assert np.array_equal(rp[k], want), f"run {j} replication {k} vs oracle"
    finally:
        for h in {id(h): h for h in handles}.values():
            h.close()


def test_batch_reports_device_errors(Bd):
    run = W.single_station(1000, 1.0, 3000.0, 0.01, 1.0, 64, 1)
    ok = W.tandem3(R=10)
    h1, h2 = Bd.EulerNet(run.net), Bd.EulerNet(ok.net)
    try:
        h1.set_option(Bd.OPT_SAMPLER_CAP, 1)
        b = Bd.Batch([h1, h2], [(0, 0.01, 1.0, 64, 1, 0), (1, ok.dt, 0.5, 10, 2, 0)])
        try:
            with pytest.raises(Bd.EulerError) as ei:
                b.run()
            assert ei.value.code == -5
        finally:
            b.close()
    finally:
        h1.close()
        h2.close()
