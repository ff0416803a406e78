"""ctypes wrapper of the C oracle (test infrastructure only).

The shared library ``oracle/liboracle.so`` is compiled by
``__graft_entry__.build()`` (or ``build_oracle()`` below) with contraction
off, so every float expression is evaluated exactly as written.
"""
from __future__ import annotations

import copy
import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

from paper_2402_13259_gb300.workloads import ARR_NONE, Network

__all__ = [
    "build_oracle", "lib", "simulate", "num_steps", "stats_split", "philox", "map_f32",
    "draw_poisson", "draw_binomial", "draw_gamma", "draw_normal", "draw_departure",
    "draw_route", "uniforms", "counters", "counters_reset", "set_cap", "COUNTER_NAMES",
    "BACKWARD", "FORWARD", "grad", "set_departure_mode", "sojourn", "sojourn_pstay", "des_simulate",
    "set_grad_center", "des_sojourn",
]

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.environ.get("EULER_ORACLE_SO") or os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "euler_oracle.c"), os.path.join(HERE, "exact_des.c")]
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]

BACKWARD, FORWARD = 0, 1

COUNTER_NAMES = [
    "units", "philox_blocks", "uniforms",
    "pois_inv", "pois_inv_iters", "pois_ptrs", "pois_ptrs_iters", "pois_ptrs_logtests",
    "bin_inv", "bin_inv_iters", "bin_btrs", "bin_btrs_iters", "bin_btrs_logtests",
    "gamma_small", "gamma_small_logs", "gamma_mt", "gamma_mt_iters", "normal_iters",
    "dep_le_m", "dep_t_gt_h", "dep_t_le_h", "route_binomials", "gather_edges",
]


def build_oracle(force: bool = False) -> str:
    if os.environ.get("EULER_ORACLE_SO"):
        return SO_PATH  # a prebuilt variant (used by the mutation test)
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "euler_oracle.h"),
                                                          os.path.join(HERE, "exact_des.h")])
    if force or not os.path.exists(SO_PATH) or os.path.getmtime(SO_PATH) < newest:
        tmp = SO_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *SOURCES, "-lm"])
        os.replace(tmp, SO_PATH)
    return SO_PATH


class _Net(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("prob", C.c_void_p),
        ("servers", C.c_void_p), ("mu", C.c_void_p), ("arr_kind", C.c_int32),
        ("w", C.c_void_p), ("a", C.c_double), ("b", C.c_double), ("period", C.c_double),
        ("phase", C.c_double), ("table", C.c_void_p), ("table_len", C.c_int32),
        ("tab_dt", C.c_double), ("N0", C.c_void_p),
        ("sv_table", C.c_void_p), ("sv_len", C.c_int32), ("sv_dt", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(SO_PATH)
        L.eo_simulate.restype = C.c_int
        L.eo_simulate.argtypes = [C.POINTER(_Net), C.c_int32, C.c_double, C.c_double, C.c_int64,
                                  C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]
        L.eo_num_steps.restype = C.c_int64
        L.eo_num_steps.argtypes = [C.c_double, C.c_double]
        L.eo_set_cap.restype = C.c_int32
        L.eo_set_cap.argtypes = [C.c_int32]
        L.eo_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.eo_map_f32.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_int64]
        L.eo_draw_poisson.argtypes = [C.c_float, C.c_uint64, C.c_int64, C.c_void_p]
        L.eo_draw_binomial.argtypes = [C.c_int32, C.c_float, C.c_uint64, C.c_int64, C.c_void_p]
        L.eo_draw_gamma.argtypes = [C.c_int32, C.c_float, C.c_uint64, C.c_int64, C.c_void_p]
        L.eo_draw_normal.argtypes = [C.c_uint64, C.c_int64, C.c_void_p]
        L.eo_draw_departure.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                        C.c_int64, C.c_void_p]
        L.eo_draw_route.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_uint64, C.c_int64,
                                    C.c_void_p]
        L.eo_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_int64, C.c_void_p]
        L.eo_counters_get.argtypes = [C.c_void_p]
        L.eo_set_departure_mode.restype = C.c_int32
        L.eo_set_departure_mode.argtypes = [C.c_int32]
        L.eo_set_grad_center.argtypes = [C.c_int32]
        L.eo_set_grad_center.restype = C.c_int32
        L.eo_grad.restype = C.c_int
        L.eo_des_simulate.argtypes = [C.POINTER(_Net), C.c_double, C.c_double, C.c_int64, C.c_uint64,
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.eo_des_sojourn.argtypes = [C.POINTER(_Net), C.c_double, C.c_double, C.c_int64, C.c_uint64,
                                     C.c_int64, C.c_int32, C.c_double, C.c_void_p, C.c_void_p]
        L.eo_sojourn.argtypes = [C.POINTER(_Net), C.c_int32, C.c_double, C.c_double, C.c_int64,
                                 C.c_uint64, C.c_int64, C.c_int32, C.c_int64, C.c_int32,
                                 C.c_void_p, C.c_void_p]
        L.eo_sojourn_pstay.argtypes = [C.c_int32, C.c_int32, C.c_int32]
        L.eo_sojourn_pstay.restype = C.c_float
        L.eo_grad.argtypes = [C.POINTER(_Net), C.c_int32, C.c_double, C.c_double, C.c_int64,
                              C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.eo_simulate_resume.restype = C.c_int
        L.eo_simulate_resume.argtypes = [C.POINTER(_Net), C.c_int32, C.c_double, C.c_double, C.c_int64,
                                         C.c_uint64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        L.eo_set_arrival_window.argtypes = [C.c_int64, C.c_int64, C.c_double]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _make_net(net: Network):
    keep = []
    a = net.arrivals
    s = _Net()
    s.n = net.n
    for name in ("row_ptr", "col", "prob", "servers", "mu"):
        arr = getattr(net, name)
        if arr.size == 0:
            arr = np.zeros(1, dtype=arr.dtype)
        keep.append(arr)
        setattr(s, name, _ptr(arr))
    s.arr_kind = a.kind
    if a.w is not None:
        keep.append(a.w)
        s.w = _ptr(a.w)
    s.a, s.b, s.period, s.phase = a.a, a.b, a.period, a.phase
    if a.table is not None:
        keep.append(a.table)
        s.table = _ptr(a.table)
        s.table_len = a.table.shape[0]
    s.tab_dt = a.tab_dt
    if net.N0 is not None:
        keep.append(net.N0)
        s.N0 = _ptr(net.N0)
    if getattr(net, "servers_schedule", None) is not None:
        tab = np.ascontiguousarray(net.servers_schedule, dtype=np.int32)
        keep.append(tab)
        s.sv_table = _ptr(tab)
        s.sv_len = tab.shape[0]
        s.sv_dt = net.servers_schedule_dt
    return s, keep


def num_steps(dt: float, T: float) -> int:
    return int(lib().eo_num_steps(dt, T))


def stats_split(stats: np.ndarray, n: int, R: int) -> Dict[str, np.ndarray]:
    st = stats[: 5 * n].reshape(n, 5)
    rp = stats[5 * n: 5 * n + 4 * R].reshape(R, 4)
    nk = stats[5 * n + 4 * R: 6 * n + 4 * R]
    return {"station": st, "rep": rp, "NK": nk}


def simulate(net: Network, scheme: int, dt: float, T: float, R: int, seed: int,
             rep_begin: int = 0, trace: bool = False, expect_ok: bool = True):
    """Run the oracle; returns dict with 'stats' (flat int64), split views, and
    optionally 'N', 'D', 'A' traces of shape [K, n, R]."""
    L = lib()
    s, keep = _make_net(net)
    n = net.n
    stats = np.zeros(6 * n + 4 * R, dtype=np.int64)
    K = num_steps(dt, T)
    tr = {}
    if trace:
        for k in ("N", "D", "A"):
            tr[k] = np.zeros((K, n, R), dtype=np.int32)
    rc = L.eo_simulate(C.byref(s), scheme, dt, T, R, seed, rep_begin, _ptr(stats),
                       _ptr(tr.get("N")), _ptr(tr.get("D")), _ptr(tr.get("A")))
    del keep
    if expect_ok and rc != 0:
        raise RuntimeError(f"oracle eo_simulate failed with code {rc}")
    out = {"rc": rc, "stats": stats, "K": K}
    out.update(stats_split(stats, n, R))
    out.update(tr)
    return out


def grad(net: Network, scheme: int, dt: float, T: float, R: int, seed: int, rep_begin: int = 0,
         scores: bool = False):
    """Likelihood-ratio gradient (see eo_grad): dict with 'grad' [2, n+3],
    'value' [2], 'var' [2, n+3] and optionally 'scores' [R, n+3]."""
    L = lib()
    s, keep = _make_net(net)
    C_ = net.n + 3
    g = np.zeros((2, C_))
    v = np.zeros(2)
    var = np.zeros((2, C_))
    sc = np.zeros((R, C_)) if scores else None
    rc = L.eo_grad(C.byref(s), scheme, dt, T, R, seed, rep_begin, _ptr(sc), _ptr(g), _ptr(v), _ptr(var))
    del keep
    if rc != 0:
        raise RuntimeError(f"oracle eo_grad failed with code {rc}")
    out = {"grad": g, "value": v, "var": var}
    if scores:
        out["scores"] = sc
    return out


def sojourn(net: Network, scheme: int, dt: float, T: float, R: int, seed: int, station: int,
            tau0: int, samples: int = 1, rep_begin: int = 0, expect_ok: bool = True):
    """Algorithm 4 on the oracle's sample paths (see eo_sojourn): dict with
    'steps' [R, samples] int32 (> 0 completed, <= 0 censored) and the paths'
    'stats' with their split views."""
    L = lib()
    s, keep = _make_net(net)
    out = np.zeros((R, samples), dtype=np.int32)
    stats = np.zeros(6 * net.n + 4 * R, dtype=np.int64)
    rc = L.eo_sojourn(C.byref(s), scheme, dt, T, R, seed, rep_begin, station, tau0, samples,
                      _ptr(out), _ptr(stats))
    del keep
    if expect_ok and rc != 0:
        raise RuntimeError(f"oracle eo_sojourn failed with code {rc}")
    res = {"rc": rc, "steps": out, "stats": stats}
    res.update(stats_split(stats, net.n, R))
    return res


def des_simulate(net: Network, dt: float, T: float, R: int, seed: int, rep_begin: int = 0,
                 trace: bool = False):
    """Exact event-by-event simulation (see exact_des.h) observed on the Euler
    grid: dict with 'stats', its split views, 'events' and optionally 'N'
    [K, n, R]."""
    L = lib()
    s, keep = _make_net(net)
    n = net.n
    K = num_steps(dt, T)
    stats = np.zeros(6 * n + 4 * R, dtype=np.int64)
    tr = np.zeros((K, n, R), dtype=np.int32) if trace else None
    ev = np.zeros(1, dtype=np.int64)
    rc = L.eo_des_simulate(C.byref(s), dt, T, R, seed, rep_begin, _ptr(stats), _ptr(tr), _ptr(ev))
    del keep
    if rc != 0:
        raise RuntimeError(f"oracle eo_des_simulate failed with code {rc}")
    out = {"stats": stats, "K": K, "events": int(ev[0])}
    out.update(stats_split(stats, n, R))
    if trace:
        out["N"] = tr
    return out


def des_sojourn(net: Network, dt: float, T: float, R: int, seed: int, station: int, t0: float,
                rep_begin: int = 0) -> np.ndarray:
    """Exact sojourn times of a tagged customer joining `station` at time t0
    in each replication (see exact_des.h): [R] doubles, -1 if not out by K dt."""
    L = lib()
    s, keep = _make_net(net)
    out = np.zeros(R, dtype=np.float64)
    rc = L.eo_des_sojourn(C.byref(s), dt, T, R, seed, rep_begin, station, t0, _ptr(out), None)
    del keep
    if rc != 0:
        raise RuntimeError(f"oracle eo_des_sojourn failed with code {rc}")
    return out


def sojourn_pstay(x: int, d: int, m: int) -> float:
    """Lemma 3's stay probability as the oracle evaluates it (float32)."""
    return float(lib().eo_sojourn_pstay(int(x), int(d), int(m)))


def simulate_resume(net: Network, scheme: int, dt: float, T: float, R: int, seed: int, tau0: int,
                    N_in: Optional[np.ndarray] = None, rep_begin: int = 0):
    """Steps tau0+1 .. K from N_in ([n, R] int32, N_tau0; None = N0), see
    eo_simulate_resume: dict with the statistics of those steps (as
    simulate()) and 'N_out' [n, R], N_K."""
    L = lib()
    s, keep = _make_net(net)
    n = net.n
    stats = np.zeros(6 * n + 4 * R, dtype=np.int64)
    nin = None if N_in is None else np.ascontiguousarray(N_in, dtype=np.int32).reshape(n, R)
    nout = np.zeros((n, R), dtype=np.int32)
    rc = L.eo_simulate_resume(C.byref(s), scheme, dt, T, R, seed, rep_begin, tau0, _ptr(nin),
                              _ptr(nout), _ptr(stats))
    del keep
    if rc != 0:
        raise RuntimeError(f"oracle eo_simulate_resume failed with code {rc}")
    out = {"stats": stats, "N_out": nout}
    out.update(stats_split(stats, n, R))
    return out


def set_arrival_window(lo: int, hi: int, factor: float):
    """Multiply the external arrival means of steps lo..hi by `factor` in
    later runs; set_arrival_window(1, 0, 1.0) switches it off."""
    lib().eo_set_arrival_window(lo, hi, factor)


def grad_coupled(net: Network, scheme: int, dt: float, T: float, R: int, seed: int, windows: int,
                 delta: float, params=None, rep_begin: int = 0):
    """Central differences under common random numbers of L_1 = dt sum N and
    L_2 = sum D with respect to theta = (mu_0..mu_{n-1}, s_0..s_{W-1}), s_w a
    factor on the external arrival means of the steps of window w, steps
    floor(wK/W)+1 .. floor((w+1)K/W).  Parameter c: the run at
    theta_c (1 + delta) minus the run at theta_c (1 - delta), same seed, per
    replication, over 2 delta theta_c; a window's runs start from N at the
    step before the window (itself from a run of the unperturbed network).
    Returns 'grad' and 'var' (variance of the mean), [2, len(params)]: the
    mean from the exact integer sum of the differences, the variance from
    S2 = sum of squares in ascending replication order."""
    n = net.n
    K = num_steps(dt, T)
    P = n + windows
    idx = list(range(P)) if params is None else [int(c) for c in params]
    g = np.zeros((2, len(idx)))
    var = np.zeros((2, len(idx)))
    for k, c in enumerate(idx):
        if c < n:
            theta = float(net.mu[c])
            runs = []
            for f in (1.0 + delta, 1.0 - delta):
                pert = copy.deepcopy(net)
                pert.mu = np.array(net.mu, dtype=np.float64)
                pert.mu[c] = theta * f
                runs.append(simulate_resume(pert, scheme, dt, T, R, seed, 0, None, rep_begin))
        else:
            theta = 1.0
            w = c - n
            lo, hi = w * K // windows + 1, (w + 1) * K // windows
            start = None
            if lo > 1:
                start = simulate_resume(net, scheme, dt, (lo - 1) * dt, R, seed, 0, None, rep_begin)["N_out"]
            runs = []
            for f in (1.0 + delta, 1.0 - delta):
                set_arrival_window(lo, hi, f)
                try:
                    runs.append(simulate_resume(net, scheme, dt, T, R, seed, lo - 1, start, rep_begin))
                finally:
                    set_arrival_window(1, 0, 1.0)
        for m in range(2):
            d = runs[0]["rep"][:, m] - runs[1]["rep"][:, m]  # int64, Q_r (m = 0) or D_r (m = 1)
            S1 = float(int(d.sum()))
            S2 = 0.0
            for x in d.tolist():
                S2 += float(x) * float(x)
            scale = (dt if m == 0 else 1.0) / (2.0 * delta * theta)
            g[m, k] = (S1 / R) * scale
            var[m, k] = ((S2 - S1 * (S1 / R)) / (R - 1)) * (scale * scale) / R if R > 1 else 0.0
    return {"grad": g, "var": var}


def set_grad_center(on: bool) -> int:
    """grad(): 1 = centred estimator mean((L - mean L) S); returns the old setting."""
    return int(lib().eo_set_grad_center(1 if on else 0))


def set_departure_mode(mode: int) -> int:
    """0 exact (Algorithm 1), 1 Eq. (1), 2 Eq. (2); returns the previous mode."""
    return int(lib().eo_set_departure_mode(mode))


def set_cap(cap: int) -> int:
    return int(lib().eo_set_cap(cap))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().eo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


_FN = {"exp": 0, "log": 1, "expm1": 2, "log1p": 3}


def map_f32(fn: str, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().eo_map_f32(_FN[fn], _ptr(x), _ptr(y), x.size)
    return y


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle sampler returned {rc}")


def draw_poisson(lam: float, seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int32)
    _check(lib().eo_draw_poisson(lam, seed, count, _ptr(out)))
    return out


def draw_binomial(n: int, p: float, seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int32)
    _check(lib().eo_draw_binomial(n, p, seed, count, _ptr(out)))
    return out


def draw_gamma(k: int, rate: float, seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    _check(lib().eo_draw_gamma(k, rate, seed, count, _ptr(out)))
    return out


def draw_normal(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    _check(lib().eo_draw_normal(seed, count, _ptr(out)))
    return out


def draw_departure(x: int, m: int, mu: float, h: float, seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int32)
    _check(lib().eo_draw_departure(x, m, mu, h, seed, count, _ptr(out)))
    return out


def draw_route(D: int, prob, seed: int, count: int) -> np.ndarray:
    p = np.ascontiguousarray(prob, dtype=np.float64)
    deg = p.size
    out = np.empty((count, deg + 1), dtype=np.int32)
    _check(lib().eo_draw_route(D, deg, _ptr(p if deg else np.zeros(1)), seed, count, _ptr(out)))
    return out


def uniforms(seed: int, purpose: int, station: int, step: int, rep: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    lib().eo_uniforms(seed, purpose, station, step, rep, count, _ptr(out))
    return out


def counters_reset():
    lib().eo_counters_reset()


def counters() -> Dict[str, int]:
    out = np.zeros(len(COUNTER_NAMES), dtype=np.int64)
    lib().eo_counters_get(_ptr(out))
    return dict(zip(COUNTER_NAMES, (int(v) for v in out)))
