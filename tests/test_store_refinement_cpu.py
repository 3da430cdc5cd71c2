"""The refinement schedules of the 16-bit stores, simulated on the CPU with the
oracle's own roundings (the products in FP64 of exactly the values the GPU
contracts): one apply of the FP16 store with its e4m3 correction term, then
one sweep of the FP16 store, reaches 1e-6; BF16 alone does not in one sweep;
the FP16 right-hand side's column scales are those of f, reused for the
residual.  CPU only; the GPU parity tests check the same numbers on the
device."""
import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W


@pytest.fixture(scope="module")
def problem():
    nx = ny = 41
    h = 1.0 / 40
    eps = W.eps_fourier(nx, ny, h, seed=1)
    rho = W.moving_charges(nx, ny, h, seed=5, steps=8)
    f = O.rhs_from_charge(nx, ny, h, eps, rho)
    Linv = O.interior_inverse(nx, ny, eps)
    return nx, ny, eps, f, Linv, (Linv @ f.T).T


def _fp16_apply(store, R, t):
    s, Q, c, C = store
    y = (s[:, None] * (Q @ R.T)).T * t[:, None]
    return y


def _corr_apply(store, R, t):
    s, Q, c, C = store
    tc = O.round_fp32(np.max(np.abs(R), axis=1) / 448.0)
    tc = np.where(tc > 0, tc, 1.0)
    r8 = O.round_e4m3(O.round_fp32(R * O.round_fp32(1.0 / tc)[:, None]))
    return (c[:, None] * (C @ r8.T)).T * (tc * t)[:, None]


def test_fp16_with_correction_one_sweep(problem):
    nx, ny, eps, f, Linv, exact = problem
    store = O.quantize_fp16_correction(Linv)
    t, R = O.quantize_cols_fp16(f)
    u = _fp16_apply(store, R, t) + _corr_apply(store, R, t)          # first apply, corrected
    e0 = O.rel_error_eq6(u, exact)
    r = O.residual(nx, ny, eps, f, u)
    Rr = O.round_fp16(r / t[:, None])                                 # the prep's scales reused
    u = u + _fp16_apply(store, Rr, t)                                 # one FP16 sweep
    e1 = O.rel_error_eq6(u, exact)
    assert 1e-6 < e0 < 1e-3
    assert e1 < 5e-7                 # 7e-8 measured: below the bench's 0.5e-6 target
    assert e1 < 1e-2 * e0


def test_bf16_alone_needs_more_than_one_sweep(problem):
    nx, ny, eps, f, Linv, exact = problem
    Q = O.round_bf16(Linv)
    u = (Q @ O.round_bf16(f).T).T
    for _ in range(1):
        u = u + (Q @ O.round_bf16(O.residual(nx, ny, eps, f, u)).T).T
    e1 = O.rel_error_eq6(u, exact)
    # the FP16 + correction schedule above is two orders of magnitude closer
    assert e1 > 1e-6
