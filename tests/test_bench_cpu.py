"""Host-side pieces of bench.py (no GPU): the launch count it claims, the
flow levels it derives, the traffic figure's guard and the workload config."""
import json

import numpy as np

import bench
from paper_2402_13259_gb300 import workloads as W


def test_num_levels_is_the_longest_path():
    assert bench.num_levels(W.layered_dag().net) == 10
    assert bench.num_levels(W.tandem3().net) == 3
    assert bench.num_levels(W.scale_dag(10, R=2).net) == 20
    # a skip edge does not shorten the longest path
    row_ptr, col, prob = W.csr_from_edges(4, [(0, 1, 0.5), (0, 3, 0.5), (1, 2, 1.0), (2, 3, 1.0)])
    net = W.Network(4, row_ptr, col, prob, np.ones(4, np.int32), np.ones(4), W.Arrivals())
    assert bench.num_levels(net) == 4


def test_launches_per_call_matches_the_graph_replays():
    # persistent form: one launch
    assert bench.launches_per_call({"form": 1}, 0, 10000, 10) == 1
    # HBM form: init + ceil(slots / 32) replays of (32 slot kernels + advance) + finish
    K, L = 10000, 10
    assert bench.launches_per_call({"form": 2}, 0, K, L) == 2 + 313 * 33      # K + 1 slots
    assert bench.launches_per_call({"form": 2}, 1, K, L) == 2 + 313 * 33      # K + L - 1 slots
    assert bench.launches_per_call({"form": 2}, 1, 20, 3) == 2 + 1 * 23       # fewer slots than a graph


def test_traffic_guard_tracks_the_kernel_sources():
    t = bench.TRAFFIC
    assert set(t) >= {"hash", "forms", "bytes_per_call"}
    h = bench.kernel_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    if t["hash"] is not None:
        assert t["forms"] == [2, 2] and t["bytes_per_call"] > 0


def test_config_names_the_workload():
    run = bench.workload()
    cfg = bench.config_dict(run, 10000, 1)
    json.dumps(cfg)
    assert "dag100" in cfg["workload"] and cfg["stations"] == 100 and cfg["steps_K"] == 10000
    assert cfg["replications_per_gpu"] == 10000 and "flushed" in cfg["l2"]


def test_reference_arm_prints_its_line():
    """--impl reference times the oracle on the host (no GPU) and prints one
    JSON line with the headline's metric and unit, its CPU description and an
    e2e object without copies."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
