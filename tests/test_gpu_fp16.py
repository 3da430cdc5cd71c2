"""GPU parity of the FP16 stores (PIDE_FP16, PIDE_FP16_FP8): the stored rows
equal the oracle's power-of-two-scaled FP16 quantisation (plus the e4m3
correction term) exactly; one apply equals the FP64 contraction of the
oracle's own roundings (s_p t_j (Q fp16(b / t)) [+ the correction]) up to
FP32 accumulation on the single-SM and SM-pair kernels, with and without the
stream-K tail; refined results reach the oracle; B = 1, the adjoint, a
tolerance-driven solve, save/load and the 3-D operator."""
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


def _b(nx, ny, h, eps, B, seed):
    return O.rhs_from_charge(nx, ny, h, eps, W.gaussian_blobs(nx, ny, h, seed, batch=B))


def _grid():
    nx, ny = 40, 33                     # n = 1178: ragged 128- and 256-row tiles
    h = 1.0 / 39
    return nx, ny, h, W.eps_fourier(nx, ny, h, seed=11)


@pytest.mark.parametrize("prec", ["fp16", "fp16_fp8"])
def test_stored_rows_equal_oracle_quantisation(prec):
    nx, ny, h, eps = _grid()
    s = _solver(nx, ny, h, eps, prec)
    n = s.n
    Linv = O.interior_inverse(nx, ny, eps)
    if prec == "fp16":
        sc, Q = O.quantize_rows_fp16(Linv)
        ref = sc[:, None] * Q
        assert s.info().precision == 6
    else:
        sc, Q, cc, C = O.quantize_fp16_correction(Linv)
        ref = sc[:, None] * Q + cc[:, None] * C
        assert s.info().precision == 7 and s.get_tuning()["corr_mask"] == 1
    for p in (0, 1, n // 2, n - 1):
        assert np.array_equal(s.inverse_row(p), ref[p]), p


def _expected_first_apply(nx, ny, eps, b, corr):
    Linv = O.interior_inverse(nx, ny, eps)
    sc, Q, cc, C = O.quantize_fp16_correction(Linv)
    t, R = O.quantize_cols_fp16(b)
    ref = (sc[:, None] * (Q @ R.T)).T * t[:, None]
    mag = (sc[:, None] * (np.abs(Q) @ np.abs(R).T)).T * t[:, None]
    if corr:
        tc = O.round_fp32(np.max(np.abs(R), axis=1) / 448.0)
        tc = np.where(tc > 0, tc, 1.0)
        r8 = O.round_e4m3(O.round_fp32(R * O.round_fp32(1.0 / tc)[:, None]))
        ref = ref + (cc[:, None] * (C @ r8.T)).T * (tc * t)[:, None]
        mag = mag + (cc[:, None] * (np.abs(C) @ np.abs(r8).T)).T * (tc * t)[:, None]
    return ref, mag


@pytest.mark.parametrize("B,pair,streamk", [(2, 1, 1), (40, 1, 1), (128, 1, 0), (300, 1, 1),
                                            (300, 1, 0), (300, 0, 1), (777, 1, 1)])
@pytest.mark.parametrize("prec", ["fp16", "fp16_fp8"])
def test_first_apply_is_exact_contraction(prec, B, pair, streamk):
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, B, seed=B + 5)
    b[0] *= 1e-20                          # a column far below the others' scale
    s = _solver(nx, ny, h, eps, prec)
    s.set_tuning(gemm_2cta=pair, gemm_streamk=streamk)
    u = s.apply(b, sweeps=0).cpu().numpy()
    ref, mag = _expected_first_apply(nx, ny, eps, b, prec == "fp16_fp8")
    err = np.abs(u - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))


def test_zero_column_and_b3():
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 3, seed=33)
    b[1] = 0.0
    s = _solver(nx, ny, h, eps, "fp16_fp8")
    u = s.apply(b, sweeps=0).cpu().numpy()
    assert not np.any(u[1])
    ref, mag = _expected_first_apply(nx, ny, eps, b, True)
    assert np.all(np.abs(u - ref) <= 2e-5 * mag + 1e-300)


@pytest.mark.parametrize("prec,mask,sweeps", [("fp16", None, 2), ("fp16_fp8", None, 1),
                                              ("fp16_fp8", 3, 1), ("fp16_fp8", 2, 2)])
def test_refined_reaches_oracle(prec, mask, sweeps):
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_lognormal(nx, ny, seed=12)
    b = _b(nx, ny, h, eps, 640, seed=13)
    s = _solver(nx, ny, h, eps, prec)
    if mask is not None:
        s.set_tuning(corr_mask=mask)
    u = s.apply(b, sweeps=sweeps).cpu().numpy()
    cols = [0, 319, 639]
    ref = O.solve(nx, ny, eps, b[cols], route="band")
    assert O.rel_error_eq6(u[cols], ref) < 1e-6


def test_boundary_values():
    """Nonzero Dirichlet values: the lift joins f before the column scale is
    taken; refined result against the oracle."""
    nx, ny, h, eps = _grid()
    rng = np.random.default_rng(7)
    g = rng.standard_normal((ny, nx))
    b = _b(nx, ny, h, eps, 200, seed=8)
    s = _solver(nx, ny, h, eps, "fp16_fp8")
    u = s.apply(b, sweeps=2, g=torch.from_numpy(g)).cpu().numpy()
    ref = O.solve(nx, ny, eps, b[[0, 199]], g)
    assert O.rel_error_eq6(u[[0, 199]], ref) < 1e-6


def test_full_size_one_sweep_sampled():
    """198^2 unknowns, B = 1024: the FP16 store with the correction in the first
    apply and one sweep, against the FP64 GPU apply (sampled columns) and the
    oracle (two columns).  The operator and the right-hand sides are the
    benchmark's own (Fourier eps and moving charges, both seed 5)."""
    nx = ny = 200
    h = 1.0 / 199
    eps = W.eps_fourier(nx, ny, h, seed=5)
    rho = W.moving_charges(nx, ny, h, seed=5, steps=1024)
    s = _solver(nx, ny, h, eps, "fp16_fp8")
    b = s.rhs_from_charge(torch.from_numpy(rho).cuda())
    u = s.apply(b, sweeps=1)
    cols = [0, 255, 256, 511, 700, 1023]
    s.close()
    s64 = _solver(nx, ny, h, eps, "fp64")
    u64 = s64.apply(b[cols])
    d = ((u[cols] - u64).abs().amax(dim=1) / u64.abs().amax(dim=1)).max().item()
    assert d < 1e-6, d
    ref = O.solve(nx, ny, eps, b[cols[:2]].cpu().numpy(), route="band")
    assert O.rel_error_eq6(u[cols[:2]].cpu().numpy(), ref) < 1e-6


def test_b1_adjoint_and_tolerance():
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 5, seed=19)
    s = _solver(nx, ny, h, eps, "fp16")
    u1 = s.apply(b[:1], sweeps=2).cpu().numpy()            # B = 1: symmetric BF16 store
    assert O.rel_error_eq6(u1, O.solve(nx, ny, eps, b[:1], route="band")) < 1e-6
    u = s.apply(b, sweeps=3)
    db, deps = s.backward(u.clone(), u, torch.from_numpy(b).cuda(), sweeps=3)
    _, db_o, deps_o = O.adjoint_gradients(nx, ny, eps, b, O.solve(nx, ny, eps, b, route="band"))
    assert np.max(np.abs(db.cpu().numpy() - db_o)) < 1e-6 * np.max(np.abs(db_o))
    assert np.max(np.abs(deps.cpu().numpy() - deps_o)) < 1e-6 * np.max(np.abs(deps_o))
    # a tolerance-driven solve stops on the device once every column is below it
    ut, info = s.apply(b, sweeps=10, tol=1e-9, want_info=True)
    assert info.converged and info.sweeps <= 6 and info.rel_residual <= 1e-9
    assert O.rel_error_eq6(ut.cpu().numpy(), O.solve(nx, ny, eps, b, route="band")) < 1e-8


def test_b1_gemv_over_the_fp16_store():
    """B = 1 through the one-term FP16 store (symv off: the GEMV with the row
    scales, FP32 right-hand side), refined to the oracle."""
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 1, seed=23)
    s = _solver(nx, ny, h, eps, "fp16")
    s.set_tuning(symv=0)
    u = s.apply(b, sweeps=3).cpu().numpy()
    assert O.rel_error_eq6(u, O.solve(nx, ny, eps, b, route="band")) < 1e-6


@pytest.mark.parametrize("prec", ["fp16", "fp16_fp8"])
def test_save_load(prec, tmp_path):
    from paper_1602_00001_gb300.binding import Solver
    nx, ny, h, eps = _grid()
    b = _b(nx, ny, h, eps, 200, seed=17)
    s = _solver(nx, ny, h, eps, prec)
    s.set_tuning(gemm_streamk=0)
    u1 = s.apply(b, sweeps=2).cpu().numpy()
    path = str(tmp_path / "inv16.bin")
    s.save(path)
    s2 = Solver.load(path)
    assert s2.info().precision == s.info().precision
    assert s2.info().store_bytes == s.info().store_bytes
    s2.set_tuning(gemm_streamk=0)
    u2 = s2.apply(b, sweeps=2).cpu().numpy()
    assert np.array_equal(u1, u2)


def test_3d_refined():
    from oracle import pide_oracle3d as O3
    from paper_1602_00001_gb300.binding import Solver3D
    nx, ny, nz = 14, 13, 12
    rng = np.random.default_rng(8)
    eps = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    n = (nx - 2) * (ny - 2) * (nz - 2)
    b = rng.standard_normal((300, n))
    s = Solver3D(nx, ny, nz, 1.0 / (nx - 1), eps, "fp16_fp8")
    u = s.apply(b, sweeps=2).cpu().numpy()
    ref = O3.solve(nx, ny, nz, eps, b[[0, 299]], route="band")
    assert np.max(np.abs(u[[0, 299]] - ref)) / np.max(np.abs(ref)) < 1e-6


@pytest.mark.parametrize("prec,nx,ny,B", [("fp16_fp8", 40, 33, 300), ("fp16", 23, 61, 5),
                                          ("fp16_fp8", 23, 61, 333), ("fp16", 5, 6, 7),
                                          ("fp16_fp8", 200, 200, 64)])
def test_cluster_prep_equals_one_cta_prep(prec, nx, ny, B):
    """The FP16 prep with a CTA cluster per column (one HBM pass, the e4m3 copy
    of R for the correction term written in the same pass) gives bit for bit
    the solution of the one-CTA prep followed by the separate e4m3 copy: with
    boundary values, with a column of zeros, for the adjoint's f = b / d, for
    an odd number of unknowns (n = 1239 at 23 x 61) and for CTA slices of 8,
    4 and 0 unknowns (n = 12 at 5 x 6)."""
    h = 1.0 / (max(nx, ny) - 1)
    eps = W.eps_lognormal(nx, ny, seed=nx * ny)
    b = _b(nx, ny, h, eps, B, seed=31)
    b[B // 2] = 0.0
    g = torch.from_numpy(np.random.default_rng(3).standard_normal((ny, nx)))
    s = _solver(nx, ny, h, eps, prec)
    s.set_tuning(gemm_streamk=0)
    outs = {}
    for pc in (1, 0):
        s.set_tuning(prep_cluster=pc)
        u = s.apply(b, sweeps=1, g=g)
        db, _ = s.backward(u.clone(), u, torch.from_numpy(b).cuda(), sweeps=1, want_deps=False)
        outs[pc] = (u, db)
    assert torch.equal(outs[1][0], outs[0][0]) and torch.equal(outs[1][1], outs[0][1])
    s.close()



def test_cluster_prep_on_a_view_8_bytes_off_16():
    """Right-hand sides that start 8 bytes past a 16-byte boundary (a view one
    element into a larger tensor): the cluster prep's solution equals the
    one-CTA prep's bit for bit."""
    nx, ny = 23, 61
    h = 1.0 / 60
    eps = W.eps_lognormal(nx, ny, seed=77)
    B = 97
    b = _b(nx, ny, h, eps, B, seed=78)
    n = b.shape[1]
    big = torch.zeros(B * n + 1, dtype=torch.float64, device="cuda")
    big[1:] = torch.from_numpy(b).cuda().reshape(-1)
    bv = big[1:].view(B, n)
    assert bv.data_ptr() % 16 == 8
    s = _solver(nx, ny, h, eps, "fp16_fp8")
    s.set_tuning(gemm_streamk=0)          # whole tiles: no atomic partial sums
    outs = {}
    for pc in (1, 0):
        s.set_tuning(prep_cluster=pc)
        outs[pc] = s.apply(bv, sweeps=1)
    assert torch.equal(outs[1], outs[0])
    s.close()
