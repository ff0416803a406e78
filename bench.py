#!/usr/bin/env python
"""Throughput of the Euler step on GB300: station-step updates per second.

Workload: the 100-station layered random DAG (10 layers x 10 stations,
m_i ~ U{100..1000}, mu_i log-uniform on [0.5, 2], utilisation <= 0.9),
10,000 replications, T = 100, dt = 0.01 (K = 10,000 steps).  One benchmark
step = one backward-scheme run plus one forward-scheme run over the whole
workload (2 x 10^10 station-step updates), through the library's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload batch512   (batched form vs one launch per network)
    python bench.py --workload rows --steps 1   (average scheme, sojourn times,
        staffing schedules, Eq. (1)/(2) departures, gradients, scale sweep)

Under torchrun each rank runs its own replication range (replication
indices rank*R ... rank*R+R-1: weak scaling, no data-path collective); at the
end of each step the ranks combine their statistics (an all-reduce of the
station rows and N_K, an all-gather of the replication rows) inside the timed
region; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "station-step updates/s per GB300 (fwd/bwd Euler), % of binding roofline"
UNIT = "station-step updates/s"
LANES_PER_SM = 128  # instruction issue: 4 schedulers x 32 lanes per clock
# DRAM bytes of one simulate call (mean of the two schemes) from one ncu
# capture of the step kernels: 11.917 MB (fused backward) and 11.938 MB
# (skewed forward) per step launch at steady state, x 10,001 and 10,009 step
# launches per call.  Valid only for the kernel sources with this hash and
# the launch forms listed; reported as null otherwise.
TRAFFIC = {"hash": "25feb6e182f56b21", "forms": [2, 2], "bytes_per_call": 0.5 * (11.917e6 * 10001 + 11.938e6 * 10009)}


def sm_count(device: int = 0) -> int:
    """Streaming multiprocessors of the device, read at run time."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def host_cpu() -> dict:
    """CPU model and logical core count of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Model Name") and v.strip():
                model = v.strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    model = v.strip()
                    break
        except OSError:
            pass
    return {"model": model or "unknown", "host_cores": os.cpu_count()}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("hbm_step.cuh", "unit.cuh", "sampling.cuh"):
        with open(os.path.join(ROOT, "paper_2402_13259_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def num_levels(net) -> int:
    """Longest-path levels of the feedforward network (the forward scheme's
    flow order)."""
    level = [0] * net.n
    indeg = [0] * net.n
    for e in range(int(net.row_ptr[-1])):
        indeg[int(net.col[e])] += 1
    order = [i for i in range(net.n) if indeg[i] == 0]
    k = 0
    while k < len(order):
        i = order[k]
        k += 1
        for e in range(int(net.row_ptr[i]), int(net.row_ptr[i + 1])):
            j = int(net.col[e])
            level[j] = max(level[j], level[i] + 1)
            indeg[j] -= 1
            if indeg[j] == 0:
                order.append(j)
    return max(level) + 1


def launches_per_call(plan, scheme: int, K: int, L: int) -> int:
    """Kernels one euler_net_simulate call launches: the persistent kernel,
    or (HBM form) init + graph replays of 32 slots of one kernel each
    (backward: K + 1 fused slots; forward: K + L - 1 skewed slots) and one
    counter advance per replay + finish."""
    if plan["form"] != 2:
        return 1
    slots = K + 1 if scheme == 0 else K + L - 1
    S = min(slots, 32)
    replays = -(-slots // S)
    return 2 + replays * (S + 1)


def workload(args=None):
    from paper_2402_13259_gb300 import workloads as W
    run = W.layered_dag()
    if args is not None and args.replications:
        run.R = args.replications
    if args is not None and args.horizon:
        run.T = args.horizon
    return run


def config_dict(run, K, world):
    return {
        "workload": f"dag100: 100-station layered random DAG (10x10), R={run.R} replications, "
                    f"T={run.T:g}, dt={run.dt:g} (K={K} steps), backward + forward scheme per step",
        "stations": run.net.n, "edges": run.net.nnz, "replications_per_gpu": run.R,
        "steps_K": K, "schemes": ["backward", "forward"],
        "state": "int32 station counts, int64 statistics, float32 samplers",
        "l2": "flushed between steps (256 MiB write)",
        "parallelism": f"replication ranges, {world} rank(s)",
    }


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(run, K_full, reps=12):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    same workload: `reps` replications x the full horizon, both schemes."""
    from oracle import oracle as O
    from paper_2402_13259_gb300 import opmodel
    per_scheme = {}
    total_units, total_t = 0, 0.0
    for scheme, name in ((0, "backward"), (1, "forward")):
        O.counters_reset()
        t0 = time.perf_counter()
        O.simulate(run.net, scheme, run.dt, run.T, reps, run.seed, rep_begin=0)
        dt = time.perf_counter() - t0
        c = O.counters()
        units = run.net.n * K_full * reps
        per_scheme[name] = {"ops_per_unit": opmodel.ops_per_unit(c),
                            "philox_blocks_per_unit": c["philox_blocks"] / max(c["units"], 1)}
        total_units += units
        total_t += dt
    # the exact event-by-event simulation of the same network, same box, same run
    des_reps = 4
    t0 = time.perf_counter()
    d = O.des_simulate(run.net, run.dt, run.T, des_reps, run.seed)
    des_t = time.perf_counter() - t0
    des = {"value": run.net.n * K_full * des_reps / des_t, "unit": UNIT + " (grid-equivalent)",
           "events_per_s": d["events"] / des_t, "cores": 1, "kind": "exact DES",
           "sample": f"{des_reps} replications over T={run.T:g} (the Euler grid's {K_full} observation "
                     f"times), single-threaded C", "seconds": des_t}
    cpu = host_cpu()
    des["cpu"] = cpu
    return {"value": total_units / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} replications x {K_full} steps x {run.net.n} stations, both schemes "
                      f"(single-threaded C oracle)", "seconds": total_t,
            "cpu": dict(cpu, used=f"1 of {cpu['host_cores']} cores"), "des": des}, per_scheme


def op_counts(run, K_full, reps=1):
    """Algorithmic operations per unit of both schemes from the oracle's event
    counters on a small sample (no timing)."""
    from oracle import oracle as O
    from paper_2402_13259_gb300 import opmodel
    per_scheme = {}
    for scheme, name in ((0, "backward"), (1, "forward")):
        O.counters_reset()
        O.simulate(run.net, scheme, run.dt, run.T, reps, run.seed, rep_begin=0)
        c = O.counters()
        per_scheme[name] = {"ops_per_unit": opmodel.ops_per_unit(c),
                            "philox_blocks_per_unit": c["philox_blocks"] / max(c["units"], 1)}
    return per_scheme


def _cpu_task(task):
    """One bounded CPU job of the CPU-baseline sweep (a worker process):
    (config, kind, scheme, rep_begin, reps) -> work and single-core seconds."""
    name, kind, scheme, rep_begin, reps = task
    from oracle import oracle as O
    run = _cpu_config(name)
    K = O.num_steps(run.dt, run.T)
    t0 = time.process_time()
    if kind == "des":
        d = O.des_simulate(run.net, run.dt, run.T, reps, run.seed, rep_begin=rep_begin)
        events = d["events"]
    else:
        O.simulate(run.net, scheme, run.dt, run.T, reps, run.seed, rep_begin=rep_begin)
        events = 0
    return name, kind, scheme, run.net.n * K * reps, events, time.process_time() - t0


def _cpu_config(name):
    from paper_2402_13259_gb300 import workloads as W
    return {"C0": W.tandem3, "C1": W.layered_dag, "C2s10": lambda: W.scale_dag(10),
            "C2s100": lambda: W.scale_dag(100), "C2s1000": lambda: W.scale_dag(1000),
            "C2s10000": lambda: W.scale_dag(10000)}[name]()


def run_cpu_baselines(args):
    """The CPU baselines of the measurement plan, on this host's cores: the
    single-threaded oracle on all of the 3-station tandem (both schemes) and
    on sampled replications of the 100-station and 2,000-station DAGs, and
    the exact DES on all of the tandem and on 100 replications of the
    100-station DAG and of the scale sweep at s = 10 and s = 100.  Every job
    is single-threaded; independent jobs run side by side in worker processes
    (one per core), and each reports its own process CPU time, so the rates
    are per core."""
    import multiprocessing as mp
    tasks = [("C0", "oracle", sc, 0, 1000) for sc in (0, 1)] + [("C0", "des", 0, 0, 1000)]
    tasks += [("C1", "oracle", sc, 100 * k, 2) for sc in (0, 1) for k in range(4)]
    for name in ("C2s10", "C2s100", "C2s1000", "C2s10000"):
        tasks += [(name, "oracle", sc, 54321, 1) for sc in (0, 1)]
    tasks += [("C1", "des", 0, 2 * k, 2) for k in range(50)]
    tasks += [("C2s10", "des", 0, 2 * k, 2) for k in range(50)]
    tasks += [("C2s100", "des", 0, k, 1) for k in range(100)]
    cpu = host_cpu()
    procs = max(1, min(os.cpu_count() or 1, args.cpu_procs or 16))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_cpu_task, tasks, chunksize=1)
    agg = {}
    for name, kind, scheme, units, events, sec in res:
        key = (name, kind, scheme if kind == "oracle" else None)
        a = agg.setdefault(key, [0, 0, 0.0, 0])
        a[0] += units
        a[1] += events
        a[2] += sec
        a[3] += 1
    from oracle import oracle as O
    for (name, kind, scheme), (units, events, sec, jobs) in sorted(agg.items(), key=str):
        run = _cpu_config(name)
        K = O.num_steps(run.dt, run.T)
        line = {"metric": f"CPU baseline {kind}: station-step updates/s per core", "impl": "cpu", "config": name,
                "kind": kind, "scheme": {0: "backward", 1: "forward", None: None}[scheme],
                "value": units / sec, "unit": UNIT + (" (grid-equivalent)" if kind == "des" else ""),
                "replications": units // (run.net.n * K), "cpu_seconds": sec,
                "cpu": dict(cpu, used=f"1 core per job, {procs} jobs side by side")}
        if kind == "des":
            line["events_per_s"] = events / sec
            line["events"] = events
        print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """--impl reference: the oracle on the host cores, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    run = workload(args)
    K = O.num_steps(run.dt, run.T)
    reps = 2
    units_per_step = 2 * run.net.n * K * reps
    for _ in range(args.warmup):
        for scheme in (0, 1):
            O.simulate(run.net, scheme, run.dt, run.T, reps, run.seed)
    t0 = time.perf_counter()
    for k in range(args.steps):
        for scheme in (0, 1):
            O.simulate(run.net, scheme, run.dt, run.T, reps, run.seed, rep_begin=reps * k)
    el = time.perf_counter() - t0
    value = units_per_step * args.steps / el
    cpu = host_cpu()
    cfg = config_dict(run, K, 1)
    cfg["replications_per_step"] = reps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{reps} replications x {K} steps x {run.net.n} stations "
                                       "per scheme per step, single-threaded C oracle",
                             "cpu": dict(cpu, used=f"1 of {cpu['host_cores']} cores")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_comparison(args):
    """512 networks of uneven size and horizon: one batched persistent launch
    (autotuned, CUDA graph) against one euler_net_simulate launch per network,
    same GB300, identical statistics required."""
    import numpy as np
    import torch
    from paper_2402_13259_gb300 import binding as Bd
    from paper_2402_13259_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    runs = W.batch_networks(512, T_scale=args.batch_T_scale, R_scale=args.batch_R_scale)
    if args.batch_subset == "small":
        # the networks a single launch cannot fill the GPU with (n R < 2^18
        # units per step): what batching is for
        runs = [r for r in runs if r.net.n * r.R < (1 << 18)]
    handles = [Bd.EulerNet(r.net) for r in runs]
    spec = [(k % 2, r.dt, r.T, r.R, r.seed, 0) for k, r in enumerate(runs)]
    units = sum(r.net.n * Bd.num_steps(r.dt, r.T) * r.R for r in runs)
    b = Bd.Batch(handles, spec)
    block = b.autotune()
    stats_b = b.alloc_stats()
    stats_s = b.alloc_stats()
    stream = torch.cuda.current_stream()

    def batched():
        b.run(stats_b, check=False)

    def per_launch():
        for h, sp, st in zip(handles, spec, stats_s):
            h.simulate(sp[0], sp[1], sp[2], sp[3], sp[4], sp[5], stats=st, check=False)

    times = {}
    for name, fn in (("batched", batched), ("per_launch", per_launch)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(f"timed_{name}")  # lets a profiler pick the timed launches
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        times[name] = e0.elapsed_time(e1) / args.steps
    b.status()
    identical = all(torch.equal(x, y) for x, y in zip(stats_b, stats_s))
    ns = sorted(r.net.n for r in runs)
    line = {"metric": "batched vs one-network-per-launch, station-step updates/s", "impl": "ours",
            "value": units / (times["batched"] / 1e3), "unit": UNIT,
            "per_launch_value": units / (times["per_launch"] / 1e3),
            "speedup": times["per_launch"] / times["batched"], "identical": identical,
            "ms_batched": times["batched"], "ms_per_launch": times["per_launch"],
            "steps": args.steps, "warmup": args.warmup, "block": block, "plan": b.info(), "n_gpus": 1,
            "config": {"workload": f"batch512: {len(runs)} of 512 layered DAGs ({args.batch_subset}), "
                                   f"n log-uniform [5,5000] (median {ns[len(ns) // 2]}), "
                                   f"T ~ U[10,200] x {args.batch_T_scale}, dt in {{0.005,0.01,0.02}}, "
                                   f"R ~ U{{100..10000}} x {args.batch_R_scale}, schemes alternate",
                       "units_per_step": units, "networks": len(runs),
                       "hbm_form_networks": sum(1 for r in runs if r.net.n * r.R >= (1 << 18))}}
    b.close()
    for h in handles:
        h.close()
    print(json.dumps(line), flush=True)
    return 0


def run_single(args):
    """--workload scale / grad: one configuration through its entry point,
    timed with CUDA events on the launching stream after one warm-up call
    with 32 replications: the scale sweep's 2,000-station DAG at --scale s
    (euler_net_simulate, both schemes), or the likelihood-ratio gradient of
    the sinusoid-arrival 100-station DAG (euler_net_grad, both schemes).
    --replications and --horizon override the configuration's R and T."""
    import torch
    from paper_2402_13259_gb300 import binding as Bd
    from paper_2402_13259_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    run = W.scale_dag(args.scale) if args.workload == "scale" else W.sinusoid_dag()
    if args.replications:
        run.R = args.replications
    if args.horizon:
        run.T = args.horizon
    n, R = run.net.n, run.R
    K = Bd.num_steps(run.dt, run.T)
    h = Bd.EulerNet(run.net)
    if args.block:
        h.set_option(Bd.OPT_BLOCK, args.block)
    stats = torch.empty(Bd.stats_len(n, R), dtype=torch.int64, device="cuda")
    for scheme, name in ((0, "backward"), (1, "forward")):
        if args.workload == "scale":
            call = lambda RR, st=None: h.simulate(scheme, run.dt, run.T, RR, run.seed, stats=st, check=False)  # noqa: E731
        else:
            call = lambda RR, st=None: h.grad(scheme, run.dt, run.T, RR, run.seed, check=False)  # noqa: E731
        call(32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            call(R, stats)
        e1.record(stream)
        torch.cuda.synchronize()
        h.status()
        ms = e0.elapsed_time(e1) / args.steps
        what = f"s={args.scale:g} 20x100 layered DAG" if args.workload == "scale" else "dag100 sinusoid, gradient"
        print(json.dumps({"metric": f"{args.workload}: station-step updates/s", "impl": "ours", "scheme": name,
                          "value": n * K * R / (ms / 1e3), "unit": UNIT, "ms_per_call": ms, "steps": args.steps,
                          "config": {"workload": f"{what}, n={n}, dt={run.dt:.4g}, T={run.T:g} (K={K}), R={R}",
                                     "plan": h.plan(scheme, R)}}), flush=True)
    h.close()
    return 0


def run_rows(args):
    """The method's other rows on the 100-station DAG at full size, each
    through its C-ABI entry point and timed with CUDA events on the launching
    stream (one warm-up call with the same dt and T first): the average
    scheme, sojourn times, a staffing schedule, the Eq. (1)/(2) departure
    samplers, likelihood-ratio gradients (100,000 replications of the
    sinusoid-arrival DAG), the coupled gradient in ten arrival windows with
    checkpointed replay (10,000 replications) and the staffing-scale sweep (2,000 stations,
    dt = 1/sqrt(s); 100,000 replications for s <= 100, 16,384 above).  One JSON line per row; bit-exact
    parity of each row is in the GPU tests."""
    import numpy as np
    import torch
    from paper_2402_13259_gb300 import binding as Bd
    from paper_2402_13259_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()

    def timed(fn, warm):
        warm()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def emit(row, units, ms, base_ms, cfg, entry, parity):
        line = {"metric": f"{row}: station-step updates/s", "impl": "ours", "row": row,
                "value": units / (ms / 1e3), "unit": UNIT, "ms_per_call": ms,
                "relative_to_simulate": (base_ms / ms) if base_ms else None, "steps": args.steps,
                "n_gpus": 1, "dtype": "f32", "data": "synthetic", "entry_point": entry,
                "parity_tests": parity, "config": cfg}
        print(json.dumps(line), flush=True)

    run = W.layered_dag()
    n, R, dt, T, seed = run.net.n, run.R, run.dt, run.T, run.seed
    K = Bd.num_steps(dt, T)
    units = n * K * R
    cfg = {"workload": f"dag100: 100-station layered DAG, R={R}, T={T:g}, dt={dt:g} (K={K})"}
    stats = torch.empty(Bd.stats_len(n, R), dtype=torch.int64, device="cuda")
    h = Bd.EulerNet(run.net)
    base = {}
    for scheme, name in ((0, "backward"), (1, "forward")):
        base[scheme] = timed(lambda: h.simulate(scheme, dt, T, R, seed, stats=stats, check=False),
                             lambda: h.simulate(scheme, dt, T, 64, seed, check=False))
        emit(f"simulate_{name}", units, base[scheme], base[scheme], cfg, "euler_net_simulate",
             "tests/test_gpu_parity.py")
    h.status()
    # f1: average scheme (both schemes + the average, 2 units per station-step)
    avg = torch.empty(Bd.stats_len(n, R), dtype=torch.float64, device="cuda")
    sb = torch.empty_like(stats)
    sf = torch.empty_like(stats)
    L = Bd.lib()

    def average(RR, out, b, f):
        Bd._check(L.euler_net_simulate_average(h._h, dt, T, RR, seed, 0, Bd.C.c_void_p(out.data_ptr()),
                                               Bd.C.c_void_p(b.data_ptr()), Bd.C.c_void_p(f.data_ptr()),
                                               Bd.C.c_void_p(stream.cuda_stream)))
    ms = timed(lambda: average(R, avg, sb, sf), lambda: average(64, avg, sb, sf))
    emit("f1_average_scheme", 2 * units, ms, base[0] + base[1], cfg, "euler_net_simulate_average",
         "tests/test_gpu_extensions.py")
    # f2: sojourn times, 4 tagged customers per replication entering station 0 at t = 50
    for scheme, name in ((0, "backward"), (1, "forward")):
        out = torch.empty((R, 4), dtype=torch.int32, device="cuda")
        ms = timed(lambda: h.sojourn(scheme, dt, T, R, seed, 0, K // 2, 4, out=out, stats=stats, check=False),
                   lambda: h.sojourn(scheme, dt, T, 64, seed, 0, K // 2, 4, check=False))
        c = dict(cfg, tagged="4 per replication, station 0, entry step K/2")
        emit(f"f2_sojourn_{name}", units, ms, base[scheme], c, "euler_net_sojourn",
             "tests/test_gpu_sojourn.py")
    h.status()
    # f4: Eq. (1) and Eq. (2) departure samplers
    for mode in (1, 2):
        h.set_option(Bd.OPT_DEPARTURE, mode)
        for scheme, name in ((0, "backward"), (1, "forward")):
            ms = timed(lambda: h.simulate(scheme, dt, T, R, seed, stats=stats, check=False),
                       lambda: h.simulate(scheme, dt, T, 64, seed, check=False))
            emit(f"f4_eq{mode}_departures_{name}", units, ms, base[scheme], cfg, "euler_net_simulate",
                 "tests/test_gpu_extensions.py")
    h.set_option(Bd.OPT_DEPARTURE, 0)
    h.status()
    h.close()
    # f3: staffing schedule, m_i(t) = m_i x (1, 1.1, 0.9, 1.2) over 25-unit intervals
    net = run.net
    fac = np.array([1.0, 1.1, 0.9, 1.2])
    net.servers_schedule = np.maximum(1, np.round(fac[:, None] * net.servers[None, :])).astype(np.int32)
    net.servers_schedule_dt = 25.0
    hs = Bd.EulerNet(net)
    for scheme, name in ((0, "backward"), (1, "forward")):
        ms = timed(lambda: hs.simulate(scheme, dt, T, R, seed, stats=stats, check=False),
                   lambda: hs.simulate(scheme, dt, T, 64, seed, check=False))
        emit(f"f3_staffing_schedule_{name}", units, ms, base[scheme],
             dict(cfg, schedule="m_i x (1, 1.1, 0.9, 1.2) per 25 time units"), "euler_net_simulate",
             "tests/test_gpu_extensions.py")
    hs.status()
    hs.close()
    net.servers_schedule = None
    # C4: likelihood-ratio gradients
    g = W.sinusoid_dag()
    hg = Bd.EulerNet(g.net)
    Kg = Bd.num_steps(g.dt, g.T)
    for scheme, name in ((0, "backward"), (1, "forward")):
        ms = timed(lambda: hg.grad(scheme, g.dt, g.T, g.R, g.seed, check=False),
                   lambda: hg.grad(scheme, g.dt, g.T, 64, g.seed, check=False))
        emit(f"c4_gradient_{name}", g.net.n * Kg * g.R, ms, None,
             {"workload": f"dag100 with sinusoid arrivals, R={g.R}, T={g.T:g}, dt={g.dt:g}",
              "gradient": "d/d(mu_1..mu_100, a, b, phase) of dt sum N and sum D"},
             "euler_net_grad", "tests/test_gpu_grad.py")
    hg.status()
    # C4, coupled variant: central differences under common random numbers in
    # the arrival scale of each of 10 time windows, each window's two runs
    # replayed from the base pass's checkpoint at the window start
    Wn, Rc = 10, 10000
    par = list(range(g.net.n, g.net.n + Wn))
    steps_run = Kg + sum(2 * (Kg - (w * Kg // Wn)) for w in range(Wn))  # base pass + replays
    steps_full = Kg + 2 * Wn * Kg  # the same without checkpoints
    for scheme, name in ((0, "backward"), (1, "forward")):
        ms = timed(lambda: hg.grad_coupled(scheme, g.dt, g.T, Rc, g.seed, Wn, 0.05, params=par, check=False),
                   lambda: hg.grad_coupled(scheme, g.dt, g.T, 64, g.seed, Wn, 0.05, params=par, check=False))
        emit(f"c4_coupled_gradient_{name}", g.net.n * steps_run * Rc, ms, None,
             {"workload": f"dag100 with sinusoid arrivals, R={Rc}, T={g.T:g}, dt={g.dt:g}",
              "gradient": f"d/d(arrival scale of {Wn} time windows) of dt sum N and sum D, "
                          "central differences, delta = 0.05, common random numbers",
              "steps_simulated": steps_run, "steps_without_checkpoints": steps_full},
             "euler_net_grad_coupled", "tests/test_gpu_resume.py")
    hg.status()
    hg.close()
    # C2: staffing-scale sweep (2,000 stations); the full 100,000 replications
    # where a call takes seconds, 16,384 (already 3.3e7 units per step) above
    for sc in (10, 100, 1000, 10000):
        rs = W.scale_dag(sc, R=100000 if sc <= 100 else 16384)
        hc = Bd.EulerNet(rs.net)
        Ks = Bd.num_steps(rs.dt, rs.T)
        st2 = torch.empty(Bd.stats_len(rs.net.n, rs.R), dtype=torch.int64, device="cuda")
        for scheme, name in ((0, "backward"), (1, "forward")):
            ms = timed(lambda: hc.simulate(scheme, rs.dt, rs.T, rs.R, rs.seed, stats=st2, check=False),
                       lambda: hc.simulate(scheme, rs.dt, rs.T, 32, rs.seed, check=False))
            emit(f"c2_scale_s{sc}_{name}", rs.net.n * Ks * rs.R, ms, None,
                 {"workload": f"20x100 layered DAG, s={sc}, dt={rs.dt:.4g}, T={rs.T:g} (K={Ks}), R={rs.R}",
                  "plan": hc.plan(scheme, rs.R)},
                 "euler_net_simulate", "tests/test_gpu_parity.py")
        hc.status()
        hc.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="dag100", choices=["dag100", "batch512", "rows", "cpu", "scale", "grad"])
    ap.add_argument("--scale", type=float, default=10000.0, help="--workload scale: the staffing scale s")
    ap.add_argument("--cpu-procs", type=int, default=16, help="--workload cpu: worker processes")
    ap.add_argument("--batch-T-scale", type=float, default=0.05,
                    help="horizon scale of the batched workload (its full 2.2e13 units take ~30 min)")
    ap.add_argument("--batch-R-scale", type=float, default=1.0)
    ap.add_argument("--batch-subset", default="all", choices=["all", "small"],
                    help="small: only the networks with n R < 2^18 units per step")
    ap.add_argument("--replications", type=int, default=0,
                    help="replications of the 100-station workload (default 10000)")
    ap.add_argument("--horizon", type=float, default=0.0, help="horizon T (default 100)")
    ap.add_argument("--form", type=int, default=0,
                    help="launch form of the 100-station workload: 0 = the planner's, 1 = persistent, 2 = HBM")
    ap.add_argument("--block", type=int, default=0,
                    help="threads per block of the 100-station workload's kernels (0 = the planner's)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch_comparison(args)
    if args.workload == "rows":
        return run_rows(args)
    if args.workload == "cpu":
        return run_cpu_baselines(args)
    if args.workload in ("scale", "grad"):
        return run_single(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2402_13259_gb300 import binding as Bd
    run = workload(args)
    K = Bd.num_steps(run.dt, run.T)
    n, R = run.net.n, run.R
    from paper_2402_13259_gb300 import sharding
    rep_begin, R = sharding.replica_range(rank, world, R, "weak")
    units_per_step = 2 * n * K * R  # per rank
    h = Bd.EulerNet(run.net)
    if args.form:
        h.set_option(Bd.OPT_FORM, args.form)
    if args.block:
        h.set_option(Bd.OPT_BLOCK, args.block)
    stream = torch.cuda.current_stream()
    stats = [torch.empty(Bd.stats_len(n, R), dtype=torch.int64, device="cuda") for _ in range(2)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")

    counts = [sharding.replica_range(r, world, run.R, "weak")[1] for r in range(world)]
    combined = [None, None]

    def one_step(events=None):
        flush.fill_(1)
        for scheme in (0, 1):
            if events is not None:
                events[scheme][0].record(stream)
            h.simulate(scheme, run.dt, run.T, R, run.seed, rep_begin, stats=stats[scheme], check=False)
            if events is not None:
                events[scheme][1].record(stream)
        if world > 1:
            # the run's one exchange: statistics over all ranks' replications
            for scheme in (0, 1):
                combined[scheme] = sharding.combine_stats_dist(stats[scheme], n, counts)

    for _ in range(args.warmup):
        one_step()
    h.status()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        one_step(ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    h.status()
    if world > 1:
        # every rank holds the whole job's statistics: its own rows in place,
        # and the station totals equal the replication totals
        for scheme in (0, 1):
            cb = combined[scheme]
            sp = Bd.split_stats(cb, n, world * R)
            assert torch.equal(sp["rep"][rank * R:(rank + 1) * R].reshape(-1), stats[scheme][5 * n:5 * n + 4 * R])
            assert int(sp["station"][:, 0].sum()) == int(sp["rep"][:, 0].sum())
    elapsed_ms = t_start.elapsed_time(t_end)
    kern_ms = [sum(ev[k][s][0].elapsed_time(ev[k][s][1]) for k in range(args.steps)) / args.steps
               for s in (0, 1)]
    if world > 1:
        t = torch.tensor([elapsed_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * units_per_step / (ms_per_step / 1e3)

    # end to end through the host-buffer entry point: network upload, both
    # schemes, statistics copied back to host memory, every step
    e2e = None
    if not args.no_e2e:
        import numpy as np
        out = [np.empty(Bd.stats_len(n, R), dtype=np.int64) for _ in range(2)]
        torch.cuda.synchronize()
        h2d = 0
        t0 = time.perf_counter()
        for k in range(args.steps):
            he = Bd.EulerNet(run.net)
            if args.form:
                he.set_option(Bd.OPT_FORM, args.form)
            if args.block:
                he.set_option(Bd.OPT_BLOCK, args.block)
            for scheme in (0, 1):
                he.simulate_host(scheme, run.dt, run.T, R, run.seed, rep_begin, out=out[scheme])
            h2d = he.h2d_bytes()
            he.close()
        e2e_s = (time.perf_counter() - t0) / args.steps
        if world > 1:  # the slowest rank's time, as for the device-timed value
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * units_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": world * h2d,
               "d2h_bytes_per_step": world * 2 * 8 * Bd.stats_len(n, R)}
    plans = {"backward": h.plan(0, R), "forward": h.plan(1, R)}
    L = num_levels(run.net)
    launches = {name: launches_per_call(plans[name], sc, K, L) for sc, name in ((0, "backward"), (1, "forward"))}
    h.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    base, per_scheme = (None, None)
    if not args.no_cpu_baseline and world == 1:
        base, per_scheme = cpu_baseline(run, K)
    elif not args.no_cpu_baseline:
        per_scheme = op_counts(run, K)  # the roofline's operation counts only
    units_launch = n * K * R
    roof = None
    if per_scheme:
        ops = [per_scheme["backward"]["ops_per_unit"] * units_launch,
               per_scheme["forward"]["ops_per_unit"] * units_launch]
        achieved = sum(ops) / (sum(kern_ms) / 1e3)
        sm_max = clk.get("sm_max_mhz") or getattr(torch.cuda.get_device_properties(local), "clock_rate", 0) / 1e3
        sms = sm_count(local)
        peak = sms * LANES_PER_SM * sm_max * 1e6
        valid = TRAFFIC["hash"] == kernel_hash() and TRAFFIC.get("forms") == [plans["backward"]["form"],
                                                                             plans["forward"]["form"]]
        hbm = plans["backward"]["form"] == 2
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                "frac": achieved / peak,
                "traffic": TRAFFIC["bytes_per_call"] if valid else None,
                "kernel": "hbm_phase_kernel (per-step kernels of one simulate call, CUDA graph)" if hbm
                          else "persistent_kernel",
                "launch": "one euler_net_simulate call per scheme (kernel time + graph launch gaps)",
                "ops_per_unit": {k: v["ops_per_unit"] for k, v in per_scheme.items()},
                "peak_note": f"{sms} SMs (device attribute) x {LANES_PER_SM} lanes x {sm_max:.0f} MHz "
                             "(nvidia-smi max SM clock; issue rate)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(run, K, world),
        "per_scheme": {"backward": {"ms_per_launch": kern_ms[0], "value": units_launch / (kern_ms[0] / 1e3)},
                       "forward": {"ms_per_launch": kern_ms[1], "value": units_launch / (kern_ms[1] / 1e3)}},
        "roofline": roof, "cpu_baseline": base, "e2e": e2e, "clocks": clk,
        "gpu_launches": (launches["backward"] + launches["forward"]) * args.steps * world,
        "plan": plans,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
