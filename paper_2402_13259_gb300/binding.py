"""Thin ctypes binding of ``libeulernet.so`` (argument marshalling only).

Every step of the simulation runs in the library's CUDA kernels; this module
only converts a :class:`workloads.Network` into the C ABI's arrays, hands
torch-allocated device buffers and the current torch stream to the library,
and maps error codes to exceptions.  There is no CPU fallback: if the library
is missing the import-time loader raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

from .workloads import Network

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeulernet.so")

BACKWARD, FORWARD = 0, 1
(OPT_FORM, OPT_TILE_REPS, OPT_BLOCK, OPT_GRID, OPT_SAMPLER_CAP, OPT_GRAPH_STEPS, OPT_PIPE_WARPS,
 OPT_WAIT_LIMIT, OPT_TEST_STALL, OPT_WAIT_SLEEP, OPT_DEPARTURE, OPT_GRAD_CENTER, OPT_HBM_CHUNK) = range(13)

ERRORS = {
    -1: "EULER_ERR_ARG", -2: "EULER_ERR_NOT_FEEDFORWARD", -3: "EULER_ERR_CUDA", -4: "EULER_ERR_OOM",
    -5: "EULER_ERR_SAMPLER_CAP", -6: "EULER_ERR_OVERFLOW", -7: "EULER_ERR_TOO_LARGE",
    -8: "EULER_ERR_STALL",
}


class EulerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Arrivals(C.Structure):
    _fields_ = [("kind", C.c_int32), ("w", C.c_void_p), ("a", C.c_double), ("b", C.c_double),
                ("period", C.c_double), ("phase", C.c_double), ("table", C.c_void_p),
                ("table_len", C.c_int32), ("tab_dt", C.c_double)]


class _Run(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("dt", C.c_double), ("T", C.c_double),
                ("replications", C.c_int64), ("seed", C.c_uint64), ("rep_begin", C.c_int64)]


_lib = None


def lib():
    """Load the library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        L.euler_net_create.argtypes = [C.POINTER(vp), i32, vp, vp, vp, vp, vp, C.POINTER(_Arrivals), vp]
        L.euler_net_create.restype = C.c_int
        L.euler_net_simulate.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, vp, vp]
        L.euler_net_simulate.restype = C.c_int
        L.euler_net_simulate_host.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, vp, vp]
        L.euler_net_simulate_host.restype = C.c_int
        L.euler_net_status.argtypes = [vp, vp]
        L.euler_net_status.restype = C.c_int
        L.euler_net_set_option.argtypes = [vp, i32, i64]
        L.euler_net_set_option.restype = C.c_int
        L.euler_net_plan.argtypes = [vp, i32, i64] + [C.POINTER(i32)] * 5
        L.euler_net_plan.restype = C.c_int
        L.euler_stats_len.argtypes = [i32, i64]
        L.euler_stats_len.restype = i64
        L.euler_num_steps.argtypes = [dbl, dbl]
        L.euler_num_steps.restype = i64
        L.euler_net_simulate_noalloc.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, vp, vp]
        L.euler_net_simulate_noalloc.restype = C.c_int
        L.euler_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.POINTER(_Run), i32]
        L.euler_batch_create.restype = C.c_int
        L.euler_batch_autotune.argtypes = [vp, vp, C.POINTER(i32)]
        L.euler_batch_autotune.restype = C.c_int
        L.euler_batch_run.argtypes = [vp, C.POINTER(vp), vp]
        L.euler_batch_run.restype = C.c_int
        L.euler_batch_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.euler_batch_info.restype = C.c_int
        L.euler_batch_status.argtypes = [vp, vp]
        L.euler_batch_status.restype = C.c_int
        L.euler_batch_destroy.argtypes = [vp]
        L.euler_batch_destroy.restype = None
        L.euler_net_batch_simulate.argtypes = [C.POINTER(vp), C.POINTER(_Run), i32, C.POINTER(vp), vp]
        L.euler_net_batch_simulate.restype = C.c_int
        L.euler_net_grad.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, vp, vp, vp, vp, vp, vp]
        L.euler_net_grad.restype = C.c_int
        L.euler_net_sojourn.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, i32, i64, i32, vp, vp, vp]
        L.euler_net_simulate_resume.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, i64, vp, vp, vp, vp]
        L.euler_net_grad_coupled.argtypes = [vp, i32, dbl, dbl, i64, u64, i64, i32, dbl, vp, i32, vp,
                                             vp, vp]
        L.euler_net_sojourn.restype = C.c_int
        L.euler_net_simulate_average.argtypes = [vp, dbl, dbl, i64, u64, i64, vp, vp, vp, vp]
        L.euler_net_simulate_average.restype = C.c_int
        L.euler_net_select_dt.argtypes = [vp, dbl]
        L.euler_net_select_dt.restype = dbl
        L.euler_net_set_servers_schedule.argtypes = [vp, vp, i32, dbl]
        L.euler_net_set_servers_schedule.restype = C.c_int
        L.euler_net_h2d_bytes.argtypes = [vp]
        L.euler_net_h2d_bytes.restype = i64
        L.euler_net_destroy.argtypes = [vp]
        L.euler_net_destroy.restype = None
        L.euler_net_last_error.argtypes = []
        L.euler_net_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise EulerError(rc, lib().euler_net_last_error().decode())


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_steps(dt: float, T: float) -> int:
    return int(lib().euler_num_steps(dt, T))


def stats_len(n: int, R: int) -> int:
    return int(lib().euler_stats_len(n, R))


def split_stats(stats, n: int, R: int) -> Dict[str, object]:
    """Views of a flat stats buffer (numpy array or torch tensor)."""
    return {"station": stats[: 5 * n].reshape(n, 5),
            "rep": stats[5 * n: 5 * n + 4 * R].reshape(R, 4),
            "NK": stats[5 * n + 4 * R: 6 * n + 4 * R]}


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class EulerNet:
    """A network resident on the current CUDA device."""

    def __init__(self, net: Network):
        L = lib()
        self.n = net.n
        a = net.arrivals
        arr = _Arrivals()
        arr.kind = a.kind
        keep = [net.row_ptr, net.col, net.prob, net.servers, net.mu]
        if a.w is not None:
            arr.w = _ptr(a.w)
            keep.append(a.w)
        arr.a, arr.b, arr.period, arr.phase = a.a, a.b, a.period, a.phase
        if a.table is not None:
            arr.table = _ptr(a.table)
            arr.table_len = a.table.shape[0]
            keep.append(a.table)
        arr.tab_dt = a.tab_dt
        h = C.c_void_p()
        rc = L.euler_net_create(C.byref(h), net.n, _ptr(net.row_ptr),
                                _ptr(net.col) if net.nnz else None,
                                _ptr(net.prob) if net.nnz else None, _ptr(net.servers), _ptr(net.mu),
                                C.byref(arr), _ptr(net.N0))
        del keep
        _check(rc)
        self._h = h
        if getattr(net, "servers_schedule", None) is not None:
            self.set_servers_schedule(net.servers_schedule, net.servers_schedule_dt)

    def set_servers_schedule(self, table, tab_dt: float):
        """Staffing schedule m_i(t) = table[j, i] (see euler_net_set_servers_schedule);
        table None clears it."""
        if table is None:
            _check(lib().euler_net_set_servers_schedule(self._h, None, 0, 1.0))
            return
        tab = np.ascontiguousarray(table, dtype=np.int32)
        _check(lib().euler_net_set_servers_schedule(self._h, _ptr(tab), tab.shape[0], float(tab_dt)))

    def close(self):
        if getattr(self, "_h", None):
            lib().euler_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def h2d_bytes(self) -> int:
        return int(lib().euler_net_h2d_bytes(self._h))

    def set_option(self, option: int, value: int):
        _check(lib().euler_net_set_option(self._h, option, value))

    def plan(self, scheme: int, R: int) -> Dict[str, int]:
        vals = [C.c_int32() for _ in range(5)]
        _check(lib().euler_net_plan(self._h, scheme, R, *[C.byref(v) for v in vals]))
        return dict(zip(["form", "tile_reps", "block", "grid", "smem"], (v.value for v in vals)))

    def simulate(self, scheme: int, dt: float, T: float, R: int, seed: int, rep_begin: int = 0,
                 stats=None, stream=None, check: bool = True):
        """Run on the device; returns the int64 stats tensor (device).  With
        check=True the stream is synchronised and device-side errors raise."""
        import torch
        n = self.n
        if stats is None:
            stats = torch.empty(stats_len(n, R), dtype=torch.int64, device="cuda")
        sp = _stream_ptr(stream)
        _check(lib().euler_net_simulate(self._h, scheme, dt, T, R, seed, rep_begin,
                                        C.c_void_p(stats.data_ptr()), C.c_void_p(sp)))
        if check:
            self.status(stream)
        return stats

    def status(self, stream=None):
        _check(lib().euler_net_status(self._h, C.c_void_p(_stream_ptr(stream))))

    def simulate_average(self, dt: float, T: float, R: int, seed: int, rep_begin: int = 0,
                         stream=None, check: bool = True):
        """Average scheme (both schemes on common random numbers): returns
        (avg float64, backward int64, forward int64) device tensors."""
        import torch
        n = self.n
        avg = torch.empty(stats_len(n, R), dtype=torch.float64, device="cuda")
        sb = torch.empty(stats_len(n, R), dtype=torch.int64, device="cuda")
        sf = torch.empty(stats_len(n, R), dtype=torch.int64, device="cuda")
        _check(lib().euler_net_simulate_average(self._h, dt, T, R, seed, rep_begin,
                                                C.c_void_p(avg.data_ptr()), C.c_void_p(sb.data_ptr()),
                                                C.c_void_p(sf.data_ptr()),
                                                C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return avg, sb, sf

    def select_dt(self, alpha: float = 0.0) -> float:
        return float(lib().euler_net_select_dt(self._h, alpha))

    def grad(self, scheme: int, dt: float, T: float, R: int, seed: int, rep_begin: int = 0,
             scores: bool = False, stats: bool = False, stream=None, check: bool = True):
        """Likelihood-ratio gradients (see euler_net_grad): dict of device
        tensors 'grad' [2, n+3], 'value' [2], 'var' [2, n+3] and optionally
        'scores' [R, n+3] and 'stats'."""
        import torch
        C_ = self.n + 3
        dev = dict(dtype=torch.float64, device="cuda")
        out = {"grad": torch.empty((2, C_), **dev), "value": torch.empty(2, **dev),
               "var": torch.empty((2, C_), **dev)}
        if scores:
            out["scores"] = torch.empty((R, C_), **dev)
        if stats:
            out["stats"] = torch.empty(stats_len(self.n, R), dtype=torch.int64, device="cuda")
        ptr = lambda k: C.c_void_p(out[k].data_ptr()) if k in out else None  # noqa: E731
        _check(lib().euler_net_grad(self._h, scheme, dt, T, R, seed, rep_begin, ptr("grad"), ptr("value"),
                                    ptr("var"), ptr("scores"), ptr("stats"),
                                    C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return out

    def simulate_resume(self, scheme: int, dt: float, T: float, R: int, seed: int, step_begin: int,
                        state_in=None, state_out: bool = False, rep_begin: int = 0, stats=None,
                        stream=None, check: bool = True):
        """Steps step_begin+1 .. K from the checkpoint state_in (int32 device
        tensor [n, R] of N_{step_begin}, or None for N0), see
        euler_net_simulate_resume: returns (stats, N_K [n, R] or None)."""
        import torch
        n = self.n
        if stats is None:
            stats = torch.empty(stats_len(n, R), dtype=torch.int64, device="cuda")
        out = torch.empty((n, R), dtype=torch.int32, device="cuda") if state_out else None
        if state_in is not None:
            assert state_in.dtype == torch.int32 and state_in.is_contiguous() and tuple(state_in.shape) == (n, R)
        _check(lib().euler_net_simulate_resume(
            self._h, scheme, dt, T, R, seed, rep_begin, step_begin,
            None if state_in is None else C.c_void_p(state_in.data_ptr()),
            None if out is None else C.c_void_p(out.data_ptr()), C.c_void_p(stats.data_ptr()),
            C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return stats, out

    def grad_coupled(self, scheme: int, dt: float, T: float, R: int, seed: int, windows: int,
                     delta: float, params=None, rep_begin: int = 0, stream=None, check: bool = True):
        """Coupled central-difference gradient with checkpointed replay (see
        euler_net_grad_coupled): dict of device tensors 'grad' and 'var',
        [2, len(params)] (params default: all n + windows)."""
        import torch
        P = self.n + windows
        idx = None if params is None else np.ascontiguousarray(params, dtype=np.int32)
        k = P if idx is None else int(idx.size)
        dev = dict(dtype=torch.float64, device="cuda")
        out = {"grad": torch.empty((2, k), **dev), "var": torch.empty((2, k), **dev)}
        _check(lib().euler_net_grad_coupled(self._h, scheme, dt, T, R, seed, rep_begin, windows, delta,
                                            _ptr(idx), k, C.c_void_p(out["grad"].data_ptr()),
                                            C.c_void_p(out["var"].data_ptr()),
                                            C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return out

    def sojourn(self, scheme: int, dt: float, T: float, R: int, seed: int, station: int, tau0: int,
                samples: int = 1, rep_begin: int = 0, out=None, stats=None, stream=None,
                check: bool = True):
        """Sojourn times of tagged customers entering `station` during step
        tau0 (see euler_net_sojourn): int32 device tensor [R, samples], the
        sojourn in steps (> 0) or minus the steps accounted when censored."""
        import torch
        if out is None:
            out = torch.empty((R, samples), dtype=torch.int32, device="cuda")
        sp = None if stats is None else C.c_void_p(stats.data_ptr())
        _check(lib().euler_net_sojourn(self._h, scheme, dt, T, R, seed, rep_begin, station, tau0, samples,
                                       C.c_void_p(out.data_ptr()), sp, C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return out

    def simulate_host(self, scheme: int, dt: float, T: float, R: int, seed: int,
                      rep_begin: int = 0, out: Optional[np.ndarray] = None, stream=None) -> np.ndarray:
        """Run with a host-memory result buffer (the library copies it back)."""
        if out is None:
            out = np.empty(stats_len(self.n, R), dtype=np.int64)
        _check(lib().euler_net_simulate_host(self._h, scheme, dt, T, R, seed, rep_begin, _ptr(out),
                                             C.c_void_p(_stream_ptr(stream))))
        return out


class Batch:
    """Many runs (network handle + run settings) in one persistent launch.

    runs: sequence of (scheme, dt, T, replications, seed, rep_begin)."""

    def __init__(self, nets, runs):
        L = lib()
        self.nets = list(nets)
        self.runs = [tuple(r) for r in runs]
        n = len(self.nets)
        handles = (C.c_void_p * n)(*[h._h.value for h in self.nets])
        rr = (_Run * n)(*[_Run(int(r[0]), float(r[1]), float(r[2]), int(r[3]), int(r[4]),
                               int(r[5]) if len(r) > 5 else 0) for r in self.runs])
        b = C.c_void_p()
        _check(L.euler_batch_create(C.byref(b), handles, rr, n))
        self._b = b

    def autotune(self, stream=None) -> int:
        blk = C.c_int32()
        _check(lib().euler_batch_autotune(self._b, C.c_void_p(_stream_ptr(stream)), C.byref(blk)))
        return blk.value

    def info(self) -> Dict[str, int]:
        """The current plan (see euler_batch_info)."""
        v = [C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()]
        _check(lib().euler_batch_info(self._b, *[C.byref(x) for x in v]))
        keys = ["hbm_networks", "hbm_min_units", "critical_path", "block", "tile_shift", "hbm_block",
                "graph_steps"]
        return dict(zip(keys, (x.value for x in v)))

    def alloc_stats(self):
        import torch
        return [torch.empty(stats_len(h.n, r[3]), dtype=torch.int64, device="cuda")
                for h, r in zip(self.nets, self.runs)]

    def run(self, stats=None, stream=None, check: bool = True):
        if stats is None:
            stats = self.alloc_stats()
        ptrs = (C.c_void_p * len(stats))(*[t.data_ptr() for t in stats])
        _check(lib().euler_batch_run(self._b, ptrs, C.c_void_p(_stream_ptr(stream))))
        if check:
            self.status(stream)
        return stats

    def status(self, stream=None):
        _check(lib().euler_batch_status(self._b, C.c_void_p(_stream_ptr(stream))))

    def close(self):
        if getattr(self, "_b", None):
            lib().euler_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _with_theta(net, theta):
    """Copy of `net` with mu = theta[:n] and sinusoid (a, b, phase) = theta[n:]."""
    import copy
    th = [float(v) for v in theta]
    net2 = copy.deepcopy(net)
    net2.mu = np.asarray(th[: net.n], dtype=np.float64)
    net2.arrivals.a, net2.arrivals.b, net2.arrivals.phase = th[net.n:]
    return net2


try:
    import torch as _torch

    class EulerMeasures(_torch.autograd.Function):
        """(E[L_1], E[L_2]) of a network as a differentiable function of
        theta = (mu_1..mu_n, a, b, phase); backward uses the likelihood-ratio
        gradient computed by the forward's kernel (no stored trajectory)."""

        @staticmethod
        def forward(ctx, theta, net, scheme, dt, T, R, seed):
            h = EulerNet(_with_theta(net, theta.detach().cpu().numpy()))
            try:
                out = h.grad(scheme, dt, T, R, seed)
            finally:
                h.close()
            ctx.save_for_backward(out["grad"].to(theta.device, theta.dtype))
            return out["value"].to(theta.device, theta.dtype)

        @staticmethod
        def backward(ctx, gout):
            (G,) = ctx.saved_tensors
            return gout @ G, None, None, None, None, None, None
except ImportError:  # pragma: no cover - torch is required for device memory
    pass
