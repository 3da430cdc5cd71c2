"""GPU parity of the BF16 store with an e4m3 correction term (PIDE_BF16_FP8):
the stored rows equal the oracle's quantisation Q + s C exactly; one apply
with the correction equals the FP64 contraction of the oracle's own roundings
(Q bf16(b) + s t (C e4m3(bf16(b) / t))) up to FP32 accumulation, on the
single-SM and SM-pair kernels, with and without the stream-K tail; refined
results reach 1e-6 against the oracle in two sweeps; save/load keeps the term."""
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


def _solver(nx, ny, h, eps, prec="bf16_fp8"):
    from paper_1602_00001_gb300.binding import Solver
    return Solver(nx, ny, h, eps, prec)


def _b(nx, ny, h, eps, B, seed):
    return O.rhs_from_charge(nx, ny, h, eps, W.gaussian_blobs(nx, ny, h, seed, batch=B))


def _grid():
    nx, ny = 40, 33                     # n = 1178: ten 128-row / five 256-row tiles, ragged
    h = 1.0 / 39
    return nx, ny, h, W.eps_fourier(nx, ny, h, seed=11)


def test_stored_rows_equal_oracle_quantisation():
    nx, ny, h, eps = _grid()
    s = _solver(nx, ny, h, eps)
    info = s.info()
    n = s.n
    assert info.precision == 5
    assert info.store_bytes >= n * info.ld * 3 + 4 * n      # BF16 Q + e4m3 C + scales
    Q, sc, C = O.quantize_bf16_correction(O.interior_inverse(nx, ny, eps))
    for p in (0, 1, n // 2, n - 1):
        assert np.array_equal(s.inverse_row(p), Q[p] + sc[p] * C[p]), p
    assert s.get_tuning()["corr_mask"] == 2                  # the default: the first sweep


def _expected_first_apply(nx, ny, eps, b):
    Q, sc, C = O.quantize_bf16_correction(O.interior_inverse(nx, ny, eps))
    R = O.round_bf16(b)
    t = O.round_fp32(np.max(np.abs(R), axis=1) / 448.0)
    t = np.where(t > 0, t, 1.0)
    r8 = O.round_e4m3(O.round_fp32(R * O.round_fp32(1.0 / t)[:, None]))
    ref = (Q @ R.T).T + (sc[:, None] * (C @ r8.T)).T * t[:, None]
    mag = (np.abs(Q) @ np.abs(R).T).T + (sc[:, None] * (np.abs(C) @ np.abs(r8).T)).T * t[:, None]
    return ref, mag


@pytest.mark.parametrize("B,pair,streamk", [(2, 1, 1), (40, 1, 1), (128, 1, 0), (300, 1, 1),
                                            (300, 1, 0), (300, 0, 1), (777, 1, 1)])
def test_first_apply_is_exact_contraction(B, pair, streamk):
    """corr_mask = 1: the first apply adds the correction term (sweeps = 0)."""
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, B, seed=B + 3)
    s = _solver(nx, ny, h, eps)
    s.set_tuning(corr_mask=1, gemm_2cta=pair, gemm_streamk=streamk)
    u = s.apply(b, sweeps=0).cpu().numpy()
    ref, mag = _expected_first_apply(nx, ny, eps, b)
    err = np.abs(u - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))


def test_mask_zero_is_the_bf16_store():
    """With no correction sweep the handle computes what a BF16 handle does
    (whole tiles only: the stream-K tail's atomic sums have no fixed order)."""
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 300, seed=9)
    s = _solver(nx, ny, h, eps)
    s.set_tuning(corr_mask=0, gemm_streamk=0)
    u1 = s.apply(b, sweeps=3).cpu().numpy()
    s2 = _solver(nx, ny, h, eps, "bf16")
    s2.set_tuning(gemm_streamk=0)
    u2 = s2.apply(b, sweeps=3).cpu().numpy()
    assert np.array_equal(u1, u2)


def test_zero_and_ragged_columns():
    """A zero right-hand side column (t = 1, all-zero e4m3 codes) stays zero and
    leaves its neighbours exact; B = 3 on the single-SM kernel."""
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 3, seed=31)
    b[1] = 0.0
    s = _solver(nx, ny, h, eps)
    s.set_tuning(corr_mask=1)
    u = s.apply(b, sweeps=0).cpu().numpy()
    assert not np.any(u[1])
    ref, mag = _expected_first_apply(nx, ny, eps, b)
    assert np.all(np.abs(u - ref) <= 2e-5 * mag + 1e-300)


@pytest.mark.parametrize("mask,sweeps", [(2, 2), (1, 2), (3, 1), (6, 2)])
def test_refined_reaches_oracle(mask, sweeps):
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_lognormal(nx, ny, seed=12)
    b = _b(nx, ny, h, eps, 640, seed=13)
    s = _solver(nx, ny, h, eps)
    s.set_tuning(corr_mask=mask)
    u = s.apply(b, sweeps=sweeps).cpu().numpy()
    cols = [0, 319, 639]
    ref = O.solve(nx, ny, eps, b[cols], route="band")
    assert O.rel_error_eq6(u[cols], ref) < 1e-6


def test_full_size_two_sweeps_sampled():
    """198^2 unknowns, B = 1024, the default mask and two sweeps against the
    FP64 GPU apply (sampled columns) and the oracle (two columns)."""
    nx = ny = 200
    h = 1.0 / 199
    eps = W.eps_fourier(nx, ny, h, seed=1)
    rho = W.moving_charges(nx, ny, h, seed=5, steps=1024)
    s = _solver(nx, ny, h, eps)
    b = s.rhs_from_charge(torch.from_numpy(rho).cuda())
    u = s.apply(b, sweeps=2)
    cols = [0, 255, 256, 511, 700, 1023]
    s.close()
    s64 = _solver(nx, ny, h, eps, "fp64")
    u64 = s64.apply(b[cols])
    d = ((u[cols] - u64).abs().amax(dim=1) / u64.abs().amax(dim=1)).max().item()
    assert d < 1e-6, d
    ref = O.solve(nx, ny, eps, b[cols[:2]].cpu().numpy(), route="band")
    assert O.rel_error_eq6(u[cols[:2]].cpu().numpy(), ref) < 1e-6


def test_save_load_keeps_the_correction(tmp_path):
    from paper_1602_00001_gb300.binding import Solver
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 200, seed=17)
    s = _solver(nx, ny, h, eps)
    s.set_tuning(gemm_streamk=0)
    u1 = s.apply(b, sweeps=2).cpu().numpy()
    path = str(tmp_path / "inv_corr.bin")
    s.save(path)
    s2 = Solver.load(path)
    assert s2.info().precision == 5 and s2.info().store_bytes == s.info().store_bytes
    s2.set_tuning(gemm_streamk=0)
    u2 = s2.apply(b, sweeps=2).cpu().numpy()
    assert np.array_equal(u1, u2)


def test_b1_and_adjoint_use_the_store():
    """B = 1 (the symmetric BF16 apply; no correction term) and the adjoint
    solve still reach the oracle's accuracy."""
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 3, seed=19)
    s = _solver(nx, ny, h, eps)
    u1 = s.apply(b[:1], sweeps=3).cpu().numpy()
    ref = O.solve(nx, ny, eps, b[:1], route="band")
    assert O.rel_error_eq6(u1, ref) < 1e-6
    ut = np.zeros_like(b)
    u = s.apply(b, sweeps=3)
    db, deps = s.backward(u - torch.from_numpy(ut).cuda(), u, torch.from_numpy(b).cuda(), sweeps=3)
    _, db_o, deps_o = O.adjoint_gradients(nx, ny, eps, b, O.solve(nx, ny, eps, b, route="band"))
    assert np.max(np.abs(db.cpu().numpy() - db_o)) < 1e-6 * np.max(np.abs(db_o))
    assert np.max(np.abs(deps.cpu().numpy() - deps_o)) < 1e-6 * np.max(np.abs(deps_o))
