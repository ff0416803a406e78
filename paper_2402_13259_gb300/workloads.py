"""Seeded synthetic inputs (networks and run settings) shared by the tests, the
benchmark, the CUDA binding and the CPU oracle.

This module holds no arithmetic of the Euler method itself: it only builds
the network description (routing CSR, server counts, service rates, arrival
rate function) from seeded numpy generators, following the workload recipes
of the benchmark configurations.  The oracle and the CUDA path each turn that
description into step-level quantities on their own.

Recipes (all seeded with ``numpy.random.default_rng``):

* ``tandem3`` -- 3-station tandem 0 -> 1 -> 2 -> exit, m_i = 50, mu_i = 1,
  lambda_0(t) = 40 (1 + 0.3 sin(2 pi t / 24)), X(0) = 0, T = 24, dt = 0.01.
* ``layered_dag`` -- L layers x W stations; m_i ~ U{100..1000}; mu_i
  log-uniform on [0.5, 2]; each non-last-layer station routes to 1-3 distinct
  uniformly chosen next-layer stations with Dirichlet(1) weights x 0.9 (exit
  0.1); the last layer exits; a next-layer station left without an in-edge is
  given one random predecessor.  Layer-0 stations get external rate
  lambda_i = 0.9 m_i mu_i; the traffic equations lambda~ = lambda + P^T
  lambda~ give the total rate into every station and a station of layer >= 1
  is restaffed to m_i = max(1, ceil(lambda~_i / (0.9 mu_i))) so that every
  utilisation is at most 0.9.
* ``scale_dag`` -- the same topology and mu with unit layer-0 base rates
  scaled by s, Halfin-Whitt staffing m_i = ceil(s l_i/mu_i + 0.5 sqrt(s
  l_i/mu_i)) (l_i the unit-scale total rate), 30 % sinusoidal modulation with
  period 24, dt = 1/sqrt(s), T = 50.
* ``batch_networks`` -- networks with station counts log-uniform on
  [5, 5000] from the layered generator with L = max(2, round(sqrt(n)/3))
  layers, horizons T ~ U[10, 200], dt in {0.005, 0.01, 0.02}, replications
  ~ U{100..10000}.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

ARR_NONE, ARR_SINUSOID, ARR_TABLE = 0, 1, 2


@dataclasses.dataclass
class Arrivals:
    """External arrival-rate function lambda_i(t).

    kind == ARR_SINUSOID: lambda_i(t) = w_i * a * (1 + b sin(2 pi t / period + phase)).
    kind == ARR_TABLE: piecewise-linear through (j*tab_dt, table[j, i]), held
    constant after the last point.
    """

    kind: int = ARR_NONE
    w: Optional[np.ndarray] = None
    a: float = 1.0
    b: float = 0.0
    period: float = 24.0
    phase: float = 0.0
    table: Optional[np.ndarray] = None
    tab_dt: float = 1.0


@dataclasses.dataclass
class Network:
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    prob: np.ndarray     # float64 [nnz]
    servers: np.ndarray  # int32 [n]
    mu: np.ndarray       # float64 [n]
    arrivals: Arrivals
    N0: Optional[np.ndarray] = None  # int32 [n]
    layer: Optional[np.ndarray] = None  # int32 [n], generator's layer index
    # optional staffing schedule m_i(t) = servers_schedule[j, i],
    # j = min(floor(t / servers_schedule_dt), J - 1)
    servers_schedule: Optional[np.ndarray] = None  # int32 [J, n]
    servers_schedule_dt: float = 1.0

    def __post_init__(self):
        self.row_ptr = np.ascontiguousarray(self.row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(self.col, dtype=np.int32)
        self.prob = np.ascontiguousarray(self.prob, dtype=np.float64)
        self.servers = np.ascontiguousarray(self.servers, dtype=np.int32)
        self.mu = np.ascontiguousarray(self.mu, dtype=np.float64)
        if self.N0 is not None:
            self.N0 = np.ascontiguousarray(self.N0, dtype=np.int32)
        a = self.arrivals
        if a.w is not None:
            a.w = np.ascontiguousarray(a.w, dtype=np.float64)
        if a.table is not None:
            a.table = np.ascontiguousarray(a.table, dtype=np.float64)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


@dataclasses.dataclass
class Run:
    """One simulation request on a network."""

    net: Network
    dt: float
    T: float
    R: int
    seed: int
    name: str = ""


def csr_from_edges(n: int, edges) -> tuple:
    """edges: iterable of (src, dst, prob) -> (row_ptr, col, prob), CSR in src order
    then insertion order."""
    rows: List[list] = [[] for _ in range(n)]
    for s, d, p in edges:
        rows[s].append((d, p))
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col, prob = [], []
    for i in range(n):
        row_ptr[i + 1] = row_ptr[i] + len(rows[i])
        for d, p in rows[i]:
            col.append(d)
            prob.append(p)
    return row_ptr, np.array(col, dtype=np.int32), np.array(prob, dtype=np.float64)


# ---------------------------------------------------------------------------
# 3-station tandem
# ---------------------------------------------------------------------------
def tandem3(R: int = 1000, seed: int = 1) -> Run:
    n = 3
    row_ptr, col, prob = csr_from_edges(n, [(0, 1, 1.0), (1, 2, 1.0)])
    w = np.array([40.0, 0.0, 0.0])
    arr = Arrivals(kind=ARR_SINUSOID, w=w, a=1.0, b=0.3, period=24.0, phase=0.0)
    net = Network(n, row_ptr, col, prob, np.full(n, 50), np.ones(n), arr,
                  layer=np.arange(n, dtype=np.int32))
    return Run(net, dt=0.01, T=24.0, R=R, seed=seed, name="tandem3")


# ---------------------------------------------------------------------------
# Layered random DAG
# ---------------------------------------------------------------------------
def _layered_topology(rng: np.random.Generator, L: int, widths: List[int]):
    starts = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
    n = int(starts[-1])
    targets = [[] for _ in range(n)]
    for l in range(L - 1):
        nxt = np.arange(starts[l + 1], starts[l + 2])
        has_in = np.zeros(len(nxt), dtype=bool)
        for i in range(starts[l], starts[l + 1]):
            deg = int(rng.integers(1, 4))
            deg = min(deg, len(nxt))
            tg = rng.choice(len(nxt), size=deg, replace=False)
            has_in[tg] = True
            targets[i] = list(nxt[tg])
        # orphans of the next layer get one random predecessor
        for j in np.nonzero(~has_in)[0]:
            i = int(rng.integers(starts[l], starts[l + 1]))
            targets[i].append(int(nxt[j]))
    edges = []
    for l in range(L - 1):
        for i in range(starts[l], starts[l + 1]):
            k = len(targets[i])
            wts = rng.dirichlet(np.ones(k)) * 0.9
            for d, p in zip(targets[i], wts):
                edges.append((i, int(d), float(p)))
    layer = np.zeros(n, dtype=np.int32)
    for l in range(L):
        layer[starts[l]:starts[l + 1]] = l
    return n, edges, layer, starts


def _traffic_rates(n: int, row_ptr, col, prob, lam_ext, layer) -> np.ndarray:
    """Total arrival rates from lambda~ = lambda + P^T lambda~ for a layered DAG,
    solved layer by layer (rows only point to later layers)."""
    tot = lam_ext.astype(np.float64).copy()
    order = np.argsort(layer, kind="stable")
    for i in order:
        for e in range(row_ptr[i], row_ptr[i + 1]):
            tot[col[e]] += tot[i] * prob[e]
    return tot


def layered_dag(L: int = 10, W: int = 10, seed: int = 2, R: int = 10000, T: float = 100.0,
                dt: float = 0.01, name: str = "dag100") -> Run:
    rng = np.random.default_rng(seed)
    widths = [W] * L
    n, edges, layer, starts = _layered_topology(rng, L, widths)
    c = rng.integers(100, 1001, size=n)
    mu = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=n))
    row_ptr, col, prob = csr_from_edges(n, edges)
    lam_ext = np.where(layer == 0, 0.9 * c * mu, 0.0)
    tot = _traffic_rates(n, row_ptr, col, prob, lam_ext, layer)
    for i in range(n):
        if layer[i] >= 1 and tot[i] > 0:
            c[i] = max(1, int(math.ceil(tot[i] / (0.9 * mu[i]))))
    arr = Arrivals(kind=ARR_SINUSOID, w=lam_ext, a=1.0, b=0.0, period=24.0, phase=0.0)
    net = Network(n, row_ptr, col, prob, c, mu, arr, layer=layer)
    return Run(net, dt=dt, T=T, R=R, seed=seed, name=name)


def scale_dag(s: float, L: int = 20, W: int = 100, seed: int = 2, R: int = 100000,
              T: float = 50.0) -> Run:
    rng = np.random.default_rng(seed)
    n, edges, layer, starts = _layered_topology(rng, L, [W] * L)
    rng.integers(100, 1001, size=n)  # keep the same draw sequence as layered_dag
    mu = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=n))
    row_ptr, col, prob = csr_from_edges(n, edges)
    base = np.where(layer == 0, 1.0, 0.0)
    tot = _traffic_rates(n, row_ptr, col, prob, base, layer)
    off = s * tot / mu
    c = np.maximum(1, np.ceil(off + 0.5 * np.sqrt(off))).astype(np.int64)
    arr = Arrivals(kind=ARR_SINUSOID, w=base * s, a=1.0, b=0.3, period=24.0, phase=0.0)
    net = Network(n, row_ptr, col, prob, c, mu, arr, layer=layer)
    return Run(net, dt=1.0 / math.sqrt(s), T=T, R=R, seed=seed, name=f"scale{int(s)}")


def batch_networks(count: int = 512, seed: int = 3, max_n: int = 5000, T_scale: float = 1.0,
                   R_scale: float = 1.0) -> List[Run]:
    """Networks of the batched workload; T_scale and R_scale shrink the
    horizons and replication counts (at least 1 replication) while keeping
    every network's structure."""
    rng = np.random.default_rng(seed)
    runs = []
    for j in range(count):
        n_target = int(round(math.exp(rng.uniform(math.log(5), math.log(max_n)))))
        L = max(2, int(round(math.sqrt(n_target) / 3)))
        W = max(1, int(round(n_target / L)))
        T = float(rng.uniform(10.0, 200.0)) * T_scale
        dt = float(rng.choice([0.005, 0.01, 0.02]))
        R = max(1, int(round(int(rng.integers(100, 10001)) * R_scale)))
        sub = layered_dag(L=L, W=W, seed=3 + j, R=R, T=T, dt=dt, name=f"batch{j}")
        runs.append(sub)
    return runs


def sinusoid_dag(theta=(1.0, 0.3, 0.0), seed: int = 2, R: int = 100000) -> Run:
    """The 100-station layered DAG with lambda_i(t) = w_i th0 (1 + th1 sin(2 pi t/24 + th2))."""
    run = layered_dag(seed=seed, R=R)
    a = run.net.arrivals
    a.kind = ARR_SINUSOID
    a.a, a.b, a.phase = float(theta[0]), float(theta[1]), float(theta[2])
    run.name = "dag100_sinusoid"
    return run


def single_station(m: int, mu: float, lam: float, dt: float, T: float, R: int, seed: int,
                   b: float = 0.0, period: float = 24.0, N0: Optional[int] = None) -> Run:
    row_ptr = np.array([0, 0], dtype=np.int32)
    arr = Arrivals(kind=ARR_SINUSOID, w=np.array([lam]), a=1.0, b=b, period=period)
    net = Network(1, row_ptr, np.zeros(0, np.int32), np.zeros(0), np.array([m]), np.array([mu]),
                  arr, N0=None if N0 is None else np.array([N0]), layer=np.zeros(1, np.int32))
    return Run(net, dt=dt, T=T, R=R, seed=seed, name="single")


def random_small_dag(rng: np.random.Generator, n: int, max_deg: int = 3, m_range=(1, 30),
                     ext_frac: float = 0.5, lam_scale: float = 5.0) -> Network:
    """A small random DAG on stations 0..n-1 (edges only to higher indices) for
    edge-case parity tests; arbitrary skips across 'layers' are allowed."""
    edges = []
    for i in range(n - 1):
        k = int(rng.integers(0, max_deg + 1))
        k = min(k, n - 1 - i)
        if k == 0:
            continue
        tg = rng.choice(np.arange(i + 1, n), size=k, replace=False)
        wts = rng.dirichlet(np.ones(k)) * rng.uniform(0.5, 1.0)
        for d, p in zip(tg, wts):
            edges.append((i, int(d), float(p)))
    row_ptr, col, prob = csr_from_edges(n, edges)
    c = rng.integers(m_range[0], m_range[1] + 1, size=n)
    mu = np.exp(rng.uniform(math.log(0.3), math.log(3.0), size=n))
    w = np.where(rng.uniform(size=n) < ext_frac, rng.uniform(0.2, 1.0, size=n) * lam_scale, 0.0)
    arr = Arrivals(kind=ARR_SINUSOID, w=w, a=1.0, b=0.4, period=7.0, phase=0.3)
    return Network(n, row_ptr, col, prob, c, mu, arr)
