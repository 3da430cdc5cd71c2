"""pide_apply_noalloc: the apply for callers that cannot allocate device
memory (it keeps its scratch in a fixed array inside the library).  Checked
through the C ABI against pide_apply on two calls in a row, plus its size
limit.  Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1602_00001_gb300 import build
    build.build()


def test_noalloc_matches_apply_twice():
    from paper_1602_00001_gb300 import binding
    lib = binding.load_library()
    n = 50
    h = 1.0 / (n - 1)
    eps = W.eps_fourier(n, n, h, seed=1)
    for prec, B in (("bf16", 5), ("fp16", 3), ("fp32", 8), ("fp64", 1)):
        s = binding.Solver(n, n, h, eps, prec)
        b = torch.from_numpy(O.rhs_from_charge(n, n, h, eps, W.gaussian_blobs(n, n, h, 9, batch=B))).cuda()
        # the scratch right-hand side is FP32: two FP64-residual sweeps take the
        # FP64 store back to FP64 accuracy
        sweeps = 2 if prec == "fp64" else 4
        u_ref = s.apply(b, sweeps=0 if prec == "fp64" else sweeps)
        stream = torch.cuda.current_stream()
        for _ in range(2):
            u = torch.full_like(b, float("nan"))
            st = lib.pide_apply_noalloc(s.handle, ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()), B, sweeps,
                                        ctypes.c_void_p(stream.cuda_stream))
            assert st == 0, lib.pide_last_error()
            torch.cuda.synchronize()
            tol = 1e-12 if prec == "fp64" else 1e-6
            assert float((u - u_ref).abs().max()) <= tol * float(u_ref.abs().max()), prec
        s.close()


def test_noalloc_rejects_oversize():
    from paper_1602_00001_gb300 import binding
    lib = binding.load_library()
    s = binding.Solver(20, 20, 1.0 / 19, None, "bf16")
    b = torch.zeros((9, s.n), dtype=torch.float64, device="cuda")
    u = torch.empty_like(b)
    st = lib.pide_apply_noalloc(s.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                9, 1, None)
    assert st == 1 and b"at most 8" in lib.pide_last_error()
    s.close()
