"""Failure detection without any GPU fault: host-side injected failures and
argument errors (CPU), and the bounded device-side wait running out on
purpose (GPU, a barrier that nothing completes, budget of a few ms)."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1602_00001_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    from paper_1602_00001_gb300 import build
    build.build()
    return binding.load_library()


def _setup(lib, eps, nx=6, ny=5):
    g = binding.Grid(nx, ny, 0.2)
    h = ctypes.c_void_p()
    e = np.ascontiguousarray(eps, dtype=np.float64)
    st = lib.pide_setup(ctypes.byref(g), e.ctypes.data_as(ctypes.c_void_p), 2, None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("bad", [np.nan, np.inf, 0.0, -1.0])
def test_bad_eps_rejected_on_host(lib, bad):
    eps = np.ones((5, 6))
    eps[2, 3] = bad
    st, h = _setup(lib, eps)
    assert st == 1 and not h.value
    assert b"eps" in lib.pide_last_error()


def test_injected_allocation_failure():
    """PIDE_FAULT_ALLOC=1 -> ENOMEM before any device work (child process so
    the environment of this one stays clean)."""
    code = (
        "import ctypes, sys; sys.path.insert(0, %r);"
        "from paper_1602_00001_gb300 import binding as B; lib = B.load_library();"
        "g = B.Grid(8, 8, 0.1); h = ctypes.c_void_p();"
        "st = lib.pide_setup(ctypes.byref(g), None, 2, None, ctypes.byref(h));"
        "print(st, lib.pide_last_error().decode())" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    out = subprocess.run([sys.executable, "-c", code], env={**os.environ, "PIDE_FAULT_ALLOC": "1"},
                         capture_output=True, text=True, timeout=120)
    st, msg = out.stdout.split(" ", 1)
    assert int(st) == 2 and "injected" in msg


def test_bad_apply_arguments(lib):
    assert lib.pide_apply(None, None, None, 4, 0, 0.0, None, None, None) == 1
    assert lib.pide_residual(None, None, None, None, 1, None) == 1
    assert lib.pide_selftest_wait_timeout(0, None) == 1


@pytest.mark.gpu
def test_bounded_wait_times_out_and_context_survives(lib):
    import torch
    assert torch.cuda.is_available()
    st = lib.pide_selftest_wait_timeout(4_000_000, None)
    assert st == 5, lib.pide_last_error()
    # the context is still usable: a small solve runs afterwards
    s = binding.Solver(12, 10, 0.1, None, "bf16")
    b = torch.ones((3, s.n), dtype=torch.float64, device="cuda")
    u = s.apply(b, sweeps=2)
    assert torch.isfinite(u).all()
    r = s.residual(b, u)
    assert float(r.abs().max()) < 1e-3
