"""pide_apply_noalloc: the refined apply for callers that cannot allocate
device memory (a fixed memory pool, a real-time loop, a plug-in that only gets
pre-sized buffers); its scratch right-hand side is a fixed array inside the
library.  Checked through the C ABI:

* one apply (no sweep) of every stored format equals the FP64 product of the
  oracle's own roundings of the inverse (with the correction term where the
  handle's mask adds it) and of the FP32 right-hand side, up to FP32
  accumulation;
* refined, it reaches the oracle's solution to 1e-6 on every stored format and
  agrees with pide_apply on the same sweep count, on two calls in a row (the
  second bit-identical to the first) that change neither torch's allocator
  nor the device's free memory;
* sizes beyond the scratch array are refused with a message.

Kept in a file collected last, so that a run stopping at its first failure has
run every other test first; it also passes alone in a fresh process."""
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


def _noalloc(lib, s, b, u, sweeps):
    stream = torch.cuda.current_stream()
    st = lib.pide_apply_noalloc(s.handle, ctypes.c_void_p(b.data_ptr()),
                                ctypes.c_void_p(u.data_ptr()), b.shape[0], sweeps,
                                ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.pide_last_error()


def _stored_operator(prec, Linv):
    """The stored inverse as the GPU holds it, written with the oracle's
    quantisers (FP64 values of the stored terms and scales)."""
    if prec == "fp64":
        return Linv
    if prec == "fp32":
        return O.round_fp32(Linv)
    if prec == "bf16":
        return O.round_bf16(Linv)
    if prec == "bf16_fp8":
        Q, c, C = O.quantize_bf16_correction(Linv)
        return Q + c[:, None] * C
    if prec == "fp16":
        s, Q = O.quantize_rows_fp16(Linv)
        return s[:, None] * Q
    if prec == "fp16_fp8":
        s, Q, c, C = O.quantize_fp16_correction(Linv)
        return s[:, None] * Q + c[:, None] * C
    s, hi, lo = O.quantize_rows_e4m3(Linv, prec == "fp8x2")
    return s[:, None] * (hi + lo)


# (format, correction mask that makes the first apply add the correction term)
@pytest.mark.parametrize("prec,mask", [("fp64", None), ("fp32", None), ("bf16", None),
                                       ("bf16_fp8", 1), ("fp16", None), ("fp16_fp8", None),
                                       ("fp8x2", None)])
def test_noalloc_one_apply_is_exact_contraction(prec, mask):
    from paper_1602_00001_gb300 import binding
    lib = binding.load_library()
    nx, ny = 31, 27
    h = 1.0 / 30
    eps = W.eps_lognormal(nx, ny, seed=4)
    s = binding.Solver(nx, ny, h, eps, prec)
    if mask is not None:
        s.set_tuning(corr_mask=mask)
    rng = np.random.default_rng(6)
    b = rng.standard_normal((5, s.n))
    bd = torch.from_numpy(b).cuda()
    u = torch.full_like(bd, float("nan"))
    _noalloc(lib, s, bd, u, 0)
    torch.cuda.synchronize()
    A = _stored_operator(prec, O.interior_inverse(nx, ny, eps))
    x = O.round_fp32(b)
    ref = x @ A.T
    mag = np.abs(x) @ np.abs(A).T
    err = np.abs(u.cpu().numpy() - ref)
    tol = 1e-12 if prec == "fp64" else 2e-5          # FP32 accumulation over <= 1 K terms
    assert np.all(err <= tol * mag + 1e-300), float(np.max(err / mag))
    s.close()


@pytest.mark.parametrize("prec,B,sweeps", [("fp64", 1, 2), ("fp32", 8, 2), ("bf16", 5, 4),
                                           ("bf16_fp8", 3, 3), ("fp16", 3, 2),
                                           ("fp16_fp8", 8, 2), ("fp8x2", 4, 4)])
def test_noalloc_refines_to_the_oracle_twice_without_allocating(prec, B, sweeps):
    from paper_1602_00001_gb300 import binding
    lib = binding.load_library()
    n = 50
    h = 1.0 / (n - 1)
    eps = W.eps_fourier(n, n, h, seed=1)
    s = binding.Solver(n, n, h, eps, prec)
    b_np = O.rhs_from_charge(n, n, h, eps, W.gaussian_blobs(n, n, h, 9, batch=B))
    ref = O.solve(n, n, eps, b_np, route="band")
    b = torch.from_numpy(b_np).cuda()
    u_apply = s.apply(b, sweeps=sweeps)
    outs = []
    for call in range(2):
        u = torch.full_like(b, float("nan"))
        torch.cuda.synchronize()
        if call == 1:
            free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        _noalloc(lib, s, b, u, sweeps)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        outs.append(u.clone())
        assert O.rel_error_eq6(u.cpu().numpy(), ref) < 1e-6, prec
    assert torch.equal(outs[0], outs[1])
    # pide_apply on the same sweep count refines to the same answer (both within
    # 1e-6 of the oracle; the first applies differ by their right-hand-side formats)
    d = ((outs[0] - u_apply).abs().amax(dim=1) / u_apply.abs().amax(dim=1)).max().item()
    assert d < 2e-6, (prec, d)
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
