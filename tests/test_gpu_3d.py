"""GPU parity of the 3-D operator (pide_setup_3d) against the 3-D oracle:
the FP64 inverse formed by block elimination over z-planes, the FP64 apply
with and without boundary values, the FP64 and double-float residuals, and
the refined low-precision applies through every apply kernel (SYMV, the
single-SM and SM-pair tensor-core GEMMs)."""
import numpy as np
import pytest

from oracle import pide_oracle3d as O3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_00001_gb300 import build, binding
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    binding.load_library()


def _solver(nx, ny, nz, eps, prec):
    from paper_1602_00001_gb300.binding import Solver3D
    return Solver3D(nx, ny, nz, 1.0 / (nx - 1), eps, prec)


def _eps(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return np.exp(0.5 * rng.standard_normal((nz, ny, nx)))


def _rel(u, ref):
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("dims", [(3, 3, 3), (5, 6, 7), (4, 3, 5), (9, 8, 7), (7, 9, 3)])
def test_fp64_apply_and_inverse_rows(dims):
    nx, ny, nz = dims
    eps = _eps(nx, ny, nz, sum(dims))
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((3, n))
    s = _solver(nx, ny, nz, eps, "fp64")
    assert s.info().dims == 3 and s.info().n == n
    u = s.apply(b).cpu().numpy()
    ref = O3.solve(nx, ny, nz, eps, b, route="dense")
    assert _rel(u, ref) < 1e-12
    Linv = O3.interior_inverse(nx, ny, nz, eps)
    for p in sorted({0, n // 2, n - 1}):
        assert np.max(np.abs(s.inverse_row(p) - Linv[p])) < 1e-13 * np.max(np.abs(Linv))


def test_boundary_values_and_fp64_residual():
    nx, ny, nz = 8, 7, 9
    eps = _eps(nx, ny, nz, 3)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(4)
    g = rng.standard_normal((nz, ny, nx))
    b = rng.standard_normal((2, n))
    s = _solver(nx, ny, nz, eps, "fp64")
    u = s.apply(b, g=torch.from_numpy(g)).cpu().numpy()
    assert _rel(u, O3.solve(nx, ny, nz, eps, b, g)) < 1e-12
    v = rng.standard_normal((2, n))
    r = s.residual(b, v).cpu().numpy()
    ref = O3.residual(nx, ny, nz, eps, b, v)
    assert np.max(np.abs(r - ref)) < 1e-14 * np.max(np.abs(v))


def _df_bound(nx, ny, nz, eps, f, u, r_exact):
    L, _, _ = O3.interior_operator(nx, ny, nz, eps)
    sc = np.abs(f) + (np.abs(L) @ np.abs(u).T).T
    return 2.0 ** -23 * np.abs(r_exact) + 2.0 ** -42 * sc + 2.0 ** -149


@pytest.mark.parametrize("dims,shape", [((10, 9, 8), 0), ((10, 9, 8), 1), ((10, 9, 8), 3),
                                        ((10, 9, 8), -1), ((26, 26, 4), 1)])
def test_double_float_residual(dims, shape):
    """The refinement's residual kernel with a z-plane of halo on each side;
    (26, 26, 4) with 8 nodes per thread needs more than 48 KB of shared
    memory (the opt-in path)."""
    nx, ny, nz = dims
    eps = _eps(nx, ny, nz, 5)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(6)
    b = 1e-3 * rng.standard_normal((5, n))
    g = rng.standard_normal((nz, ny, nx))
    ref = O3.solve(nx, ny, nz, eps, b, g, route="band")
    u = ref * (1 + 1e-5 * rng.standard_normal(ref.shape))
    f = b + O3.boundary_lift(nx, ny, nz, eps, g)[None, :]
    r_exact = O3.residual(nx, ny, nz, eps, f, u)
    s = _solver(nx, ny, nz, eps, "bf16")
    s.set_tuning(resid_shape=shape)
    r = s.residual_df(b, u, g).cpu().numpy().astype(np.float64)
    bound = _df_bound(nx, ny, nz, eps, f, u, r_exact)
    assert np.all(np.abs(r - r_exact) <= bound), float(np.max(np.abs(r - r_exact) / bound))


@pytest.mark.parametrize("prec,B,pair", [("bf16", 1, 1), ("bf16", 40, 1), ("bf16", 300, 1),
                                         ("bf16", 300, 0), ("fp8x2", 64, 1)])
def test_refined_low_precision(prec, B, pair):
    nx, ny, nz = 14, 13, 12
    eps = _eps(nx, ny, nz, 7)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(8)
    b = rng.standard_normal((B, n))
    g = 0.1 * rng.standard_normal((nz, ny, nx))
    s = _solver(nx, ny, nz, eps, prec)
    s.set_tuning(gemm_2cta=pair)
    u = s.apply(b, sweeps=8, g=torch.from_numpy(g)).cpu().numpy()
    cols = sorted({0, B // 2, B - 1})
    ref = O3.solve(nx, ny, nz, eps, b[cols], g, route="band")
    assert _rel(u[cols], ref) < 1e-6


def test_stream_and_charge():
    from paper_1602_00001_gb300.binding import Solver3D
    nx, ny, nz = 12, 11, 10
    h = 1.0 / (nx - 1)
    eps = _eps(nx, ny, nz, 9)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(10)
    rho = rng.standard_normal((700, n))
    s = Solver3D(nx, ny, nz, h, eps, "bf16")
    u = s.solve_stream(rho, chunk=256, sweeps=6, charge=True)
    b = O3.rhs_from_charge(nx, ny, nz, h, eps, rho[[0, 255, 256, 699]])
    ref = O3.solve(nx, ny, nz, eps, b, route="band")
    assert _rel(u[[0, 255, 256, 699]], ref) < 1e-6


def test_adjoint_3d():
    """dLoss/db and dLoss/deps over the six faces against the 3-D oracle's
    adjoint (itself pinned by central differences)."""
    nx, ny, nz = 7, 6, 8
    eps = _eps(nx, ny, nz, 13)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    rng = np.random.default_rng(14)
    b = rng.standard_normal((3, n))
    ut = rng.standard_normal((3, n))
    u_o, db_o, deps_o = O3.adjoint_gradients(nx, ny, nz, eps, b, np.zeros_like(b))
    u_o, db_o, deps_o = O3.adjoint_gradients(nx, ny, nz, eps, b, u_o - ut)
    for prec, sweeps, tol in (("fp64", 0, 1e-11), ("bf16", 6, 1e-6)):
        s = _solver(nx, ny, nz, eps, prec)
        u = s.apply(b, sweeps=sweeps)
        db, deps = s.backward(u - torch.from_numpy(ut).cuda(), u, torch.from_numpy(b).cuda(),
                              sweeps=sweeps)
        assert deps.shape == (nz, ny, nx)
        assert _rel(db.cpu().numpy(), db_o) < tol
        assert _rel(deps.cpu().numpy(), deps_o) < tol


def test_save_load_and_unsupported(tmp_path):
    from paper_1602_00001_gb300.binding import PideError, Solver, apply_batched
    nx, ny, nz = 6, 5, 7
    eps = _eps(nx, ny, nz, 15)
    s = _solver(nx, ny, nz, eps, "bf16")
    rng = np.random.default_rng(16)
    b = rng.standard_normal((40, s.n))
    u1 = s.apply(b, sweeps=5).cpu().numpy()
    path = str(tmp_path / "inv3d.bin")
    s.save(path)
    s2 = Solver.load(path)
    assert s2.nz == nz and s2.n == s.n and s2.info().dims == 3
    u2 = s2.apply(b, sweeps=5).cpu().numpy()
    assert _rel(u2, u1) < 1e-12
    bb = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(PideError):
        apply_batched([s], [bb], [torch.zeros_like(bb)])
