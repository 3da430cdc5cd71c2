"""GPU parity of the double-float refinement residual and prep.

The refinement residual r = f - L u of Eq. (3) is evaluated on the integer and
FP32 pipes: each FP64 input split into two floats (47 significant bits), the
stencil in error-free float arithmetic.  Its error bound, written in the
tests: |r_gpu - r| <= 2^-23 |r| (the FP32 output) + 2^-42 s_p + 2^-149, with
s_p = |f_p| + |u_p| + sum_q w_pq |u_q| (the split inputs' 2^-46 relative
rounding, four products and sums of them, and a margin of 4x); 2^-149 is the
smallest FP32 subnormal.  The exact r is the oracle's FP64 band residual.
"""
import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_00001_gb300 import build, binding
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    binding.load_library()


def _solver(nx, ny, h, eps, prec):
    from paper_1602_00001_gb300.binding import Solver
    return Solver(nx, ny, h, eps, prec)


def _bound(nx, ny, eps, f, u, r_exact):
    L, _, _ = O.interior_operator(nx, ny, eps)
    s = np.abs(f) + (np.abs(L) @ np.abs(u).T).T      # |L| = I + |W|
    return 2.0 ** -23 * np.abs(r_exact) + 2.0 ** -42 * s + 2.0 ** -149


@pytest.mark.parametrize("with_g,shape", [(False, 0), (True, 0), (True, 1), (False, 2),
                                           (True, 3)])
def test_residual_df_near_solution(with_g, shape):
    """u close to the solution (the refinement's regime): r is ~1e-5 of u,
    so the stencil sum cancels five orders of magnitude.  Every launch shape
    of the shared-memory kernel (tiles of 1024 or 2048 nodes: several tiles
    and a ragged last one here)."""
    nx, ny = 77, 69
    h = 1.0 / 76
    eps = W.eps_lognormal(nx, ny, seed=21)
    rng = np.random.default_rng(22)
    B = 7
    rho = W.gaussian_blobs(nx, ny, h, 23, batch=B)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    g = rng.standard_normal((ny, nx)) if with_g else None
    lift = O.boundary_lift(nx, ny, eps, g) if with_g else np.zeros(b.shape[1])
    ref = O.solve(nx, ny, eps, b, g)
    u = ref * (1.0 + 1e-5 * rng.standard_normal(ref.shape))
    f = b + lift[None, :]
    r_exact = O.residual(nx, ny, eps, f, u)
    s = _solver(nx, ny, h, eps, "bf16")
    s.set_tuning(resid_shape=shape)
    r = s.residual_df(b, u, g).cpu().numpy().astype(np.float64)
    bound = _bound(nx, ny, eps, f, u, r_exact)
    assert np.all(np.abs(r - r_exact) <= bound), float(np.max(np.abs(r - r_exact) / bound))
    # the FP64 residual entry point agrees with the oracle to FP64 rounding
    if not with_g:
        r64 = s.residual(b, u).cpu().numpy()
        assert np.max(np.abs(r64 - r_exact)) <= 1e-13 * np.max(np.abs(u))


@pytest.mark.parametrize("pf", [0, 1, 3, 4, 1000])
def test_residual_df_prefetch_distance_changes_no_bit(pf):
    """The L2 prefetch of the tile pf column pairs ahead (7 columns: 4 pairs,
    the last a single column; 3 prefetches that single column, 4 and 1000
    nothing) moves no result bit."""
    nx, ny = 77, 69
    h = 1.0 / 76
    eps = W.eps_lognormal(nx, ny, seed=24)
    rng = np.random.default_rng(25)
    b = O.rhs_from_charge(nx, ny, h, eps, W.gaussian_blobs(nx, ny, h, 26, batch=7))
    ref = O.solve(nx, ny, eps, b)
    u = ref * (1.0 + 1e-5 * rng.standard_normal(ref.shape))
    s = _solver(nx, ny, h, eps, "bf16")
    assert s.get_tuning()["resid_prefetch"] == 4            # the default
    s.set_tuning(resid_prefetch=0)
    r0 = s.residual_df(b, u).cpu().numpy()
    s.set_tuning(resid_prefetch=pf)
    r = s.residual_df(b, u).cpu().numpy()
    assert np.array_equal(r, r0)
    r_exact = O.residual(nx, ny, eps, b, u)
    bound = _bound(nx, ny, eps, b, u, r_exact)
    assert np.all(np.abs(r.astype(np.float64) - r_exact) <= bound)


def test_residual_df_wide_grid_register_kernel():
    """A grid row longer than the shared-memory halo allows (1028 interior
    nodes per row): the register kernel, with clamped neighbour loads."""
    nx, ny = 1030, 4
    h = 1.0 / 1029
    eps = W.eps_lognormal(nx, ny, seed=30)
    rng = np.random.default_rng(31)
    n = (nx - 2) * (ny - 2)
    u = rng.standard_normal((3, n)).cumsum(axis=1) * 1e-2
    b = 1e-3 * rng.standard_normal((3, n))
    g = rng.standard_normal((ny, nx))
    f = b + O.boundary_lift(nx, ny, eps, g)[None, :]
    r_exact = O.residual(nx, ny, eps, f, u)
    s = _solver(nx, ny, h, eps, "bf16")
    r = s.residual_df(b, u, g).cpu().numpy().astype(np.float64)
    bound = _bound(nx, ny, eps, f, u, r_exact)
    assert np.all(np.abs(r - r_exact) <= bound), float(np.max(np.abs(r - r_exact) / bound))


def test_residual_df_special_values():
    """Zeros (split exactly), values below the split's range (|x| < 2^-103:
    the node falls back to the FP64 formula), values near the top of the
    float range, and columns that mix them."""
    nx, ny = 19, 23
    h = 1.0 / 18
    eps = W.eps_lognormal(nx, ny, seed=24)
    n = (nx - 2) * (ny - 2)
    rng = np.random.default_rng(25)
    u = rng.standard_normal((6, n))
    b = rng.standard_normal((6, n))
    u[0] = 0.0
    b[0] = 0.0                                   # all zero: r = 0 exactly
    u[1][::3] = 0.0                              # scattered exact zeros
    b[1][1::4] = 0.0
    u[2] *= 1e-33                                # below 2^-103 everywhere: FP64 route
    b[2] *= 1e-33
    u[3] *= 1e36                                 # in range, near 2^128
    b[3] *= 1e36
    mask = rng.random(n) < 0.5                   # half tiny, half O(1)
    u[4][mask] *= 1e-40
    b[4][~mask] *= 1e-35
    u[5] = -np.abs(u[5]) * 2.0 ** -100           # just above the split's lower limit
    b[5] = np.abs(b[5]) * 2.0 ** -100
    r_exact = O.residual(nx, ny, eps, b, u)
    s = _solver(nx, ny, h, eps, "bf16")
    r = s.residual_df(b, u).cpu().numpy().astype(np.float64)
    assert np.all(r[0] == 0.0)
    bound = _bound(nx, ny, eps, b, u, r_exact)
    assert np.all(np.abs(r - r_exact) <= bound), float(np.max(np.abs(r - r_exact) / bound))


@pytest.mark.parametrize("prec,B,sweeps", [("bf16", 64, 6), ("bf16", 257, 6),
                                           ("fp8x2", 64, 10), ("bf16", 1, 3)])
def test_refined_with_df_residual(prec, B, sweeps):
    """The refined apply with the double-float residual and prep reaches the
    oracle's solution like the FP64-residual run, with boundary values."""
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_fourier(nx, ny, h, seed=1)
    rng = np.random.default_rng(26)
    rho = W.gaussian_blobs(nx, ny, h, 27, batch=B)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    g = 0.1 * rng.standard_normal((ny, nx))
    ref = O.solve(nx, ny, eps, b, g, route="band")
    s = _solver(nx, ny, h, eps, prec)
    assert s.get_tuning()["resid_emul"] == 1
    u1 = s.apply(b, sweeps=sweeps, g=torch.from_numpy(g)).cpu().numpy()
    s.set_tuning(resid_emul=0)
    u0 = s.apply(b, sweeps=sweeps, g=torch.from_numpy(g)).cpu().numpy()
    e1, e0 = O.rel_error_eq6(u1, ref), O.rel_error_eq6(u0, ref)
    assert e1 < 1e-6 and e0 < 1e-6, (e1, e0)
    assert O.rel_error_eq6(u1, u0) < 1e-7


def test_prep_df_with_lift_is_exact_contraction():
    """One apply (no refinement) with boundary values: the BF16 right-hand
    side is bf16(b + lift) rounded to nearest from the FP64 sum, so the result
    is the FP64 contraction of the oracle's own roundings up to FP32 accumulation."""
    nx, ny = 40, 33
    h = 1.0 / 39
    eps = W.eps_fourier(nx, ny, h, seed=11)
    rng = np.random.default_rng(28)
    B = 40
    rho = W.gaussian_blobs(nx, ny, h, 29, batch=B)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    g = rng.standard_normal((ny, nx))
    f = b + O.boundary_lift(nx, ny, eps, g)[None, :]
    s = _solver(nx, ny, h, eps, "bf16")
    u = s.apply(b, sweeps=0, g=torch.from_numpy(g)).cpu().numpy()
    Q = O.round_bf16(O.interior_inverse(nx, ny, eps))
    fq = O.round_bf16(f)
    ref, mag = (Q @ fq.T).T, (np.abs(Q) @ np.abs(fq).T).T
    assert np.all(np.abs(u - ref) <= 2e-5 * mag + 1e-300)
