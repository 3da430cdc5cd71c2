"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: the plain FP64 path within 1e-12 (Eq. 6 relative error, worst
column); the refined low-precision paths within 1e-6; single low-precision
applies against the oracle's contraction of the same rounded operands within
a bound derived from FP32 accumulation.
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


def _b(nx, ny, h, eps, B, seed):
    rho = W.gaussian_blobs(nx, ny, h, seed, batch=B)
    return O.rhs_from_charge(nx, ny, h, eps, rho)


GRIDS = [(3, 3), (3, 7), (7, 3), (5, 5), (12, 9), (21, 21), (34, 27)]


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("B", [1, 2, 5, 9, 70])
def test_fp64_apply_matches_oracle(nx, ny, B):
    h = 1.0 / (max(nx, ny) - 1)
    eps = W.eps_lognormal(nx, ny, seed=nx * 31 + ny)
    b = W.random_interior(nx, ny, seed=B, batch=B)
    s = _solver(nx, ny, h, eps, "fp64")
    u = s.apply(b).cpu().numpy()
    ref = O.solve(nx, ny, eps, b)
    assert O.rel_error_eq6(u, ref) < 1e-12


def test_fp64_inverse_rows_match_oracle():
    nx, ny = 14, 11
    eps = W.eps_fourier(nx, ny, 1.0 / 13, seed=2)
    s = _solver(nx, ny, 1.0 / 13, eps, "fp64")
    Linv = O.interior_inverse(nx, ny, eps)
    for p in [0, 5, s.n // 2, s.n - 1]:
        row = s.inverse_row(p)
        assert np.max(np.abs(row - Linv[p])) < 1e-13 * np.max(np.abs(Linv))


def test_fig3_grid_eps1():
    """nx=3, ny=5 at eps=1 (Fig. 3): three unknowns."""
    s = _solver(3, 5, 0.25, None, "fp64")
    b = np.array([[1.0, 2.0, 3.0]])
    u = s.apply(b).cpu().numpy()
    A = O.assemble_full(3, 5)
    uf = O.lu_inverse(A) @ O.full_rhs(3, 5, b)[0]
    assert np.max(np.abs(u[0] - uf[[4, 7, 10]])) < 1e-15


def test_residual_matches_oracle():
    nx, ny = 23, 17
    h = 1.0 / 22
    eps = W.eps_lognormal(nx, ny, seed=5)
    s = _solver(nx, ny, h, eps, "fp64")
    rng = np.random.default_rng(1)
    b = rng.standard_normal((3, s.n))
    u = rng.standard_normal((3, s.n))
    r = s.residual(b, u).cpu().numpy()
    ref = O.residual(nx, ny, eps, b, u)
    assert np.max(np.abs(r - ref)) < 1e-14 * np.max(np.abs(ref))


def test_rhs_from_charge_matches_oracle():
    nx, ny = 19, 15
    h = 1.0 / 18
    eps = W.eps_fourier(nx, ny, h, seed=3)
    s = _solver(nx, ny, h, eps, "fp64")
    rho = W.gaussian_blobs(nx, ny, h, seed=4, batch=2)
    b = s.rhs_from_charge(rho).cpu().numpy()
    assert np.max(np.abs(b - O.rhs_from_charge(nx, ny, h, eps, rho))) <= 1e-15 * np.max(np.abs(b))


def test_nonzero_boundary_values():
    """Fig. 3's boundary rows carry boundary values: lifting on the GPU."""
    nx, ny = 16, 12
    h = 1.0 / 15
    eps = W.eps_lognormal(nx, ny, seed=6)
    rng = np.random.default_rng(7)
    g = rng.standard_normal((ny, nx))
    b = rng.standard_normal((2, (nx - 2) * (ny - 2)))
    s = _solver(nx, ny, h, eps, "fp64")
    u = s.apply(b, g=torch.from_numpy(g)).cpu().numpy()
    ref = O.solve(nx, ny, eps, b, g)
    assert O.rel_error_eq6(u, ref) < 1e-12


# ----------------------------------------------------------- low-precision contraction


def _oracle_lowprec_apply(nx, ny, eps, b, store_round, rhs_round):
    """Q(L^-1) q(b) in FP64 with the operands rounded like the GPU stores them."""
    Q = store_round(O.interior_inverse(nx, ny, eps))
    f = rhs_round(b)
    return (Q @ f.T).T, (np.abs(Q) @ np.abs(f).T).T


@pytest.mark.parametrize("B", [1, 3, 8, 9, 40, 64, 65, 130, 300])
def test_bf16_single_apply_is_exact_contraction(B):
    """One apply (no refinement) equals the FP64 contraction of the same
    bf16-rounded inverse and right-hand side up to FP32 accumulation.  B up
    to the GEMV limit (default 1) takes the GEMV (FP32 right-hand side),
    larger B the tcgen05 GEMM (BF16 right-hand side); B <= 8 is checked on
    both by moving the limit."""
    nx, ny = 40, 33
    h = 1.0 / 39
    eps = W.eps_fourier(nx, ny, h, seed=11)
    b = _b(nx, ny, h, eps, B, seed=B)
    s = _solver(nx, ny, h, eps, "bf16")
    s.set_tuning(symv=0)          # B = 1 through the full stored L^-1 here
    # B > 128: the SM-pair kernel (default) and the single-SM kernel
    for limit, pair in ([(1, 1), (8, 1)] if B <= 8 else [(1, 1), (1, 0)] if B > 128 else [(1, 1)]):
        s.set_tuning(gemv_max_b=limit, gemm_2cta=pair)
        u = s.apply(b, sweeps=0).cpu().numpy()
        rhs_round = O.round_fp32 if B <= limit else O.round_bf16
        ref, mag = _oracle_lowprec_apply(nx, ny, eps, b, O.round_bf16, rhs_round)
        err = np.abs(u - ref)
        assert np.all(err <= 2e-5 * mag + 1e-300), (limit, pair, float(np.max(err / mag)))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("B", [1, 9, 64, 257])
def test_refined_reaches_1e6(prec, B):
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_fourier(nx, ny, h, seed=1)
    b = _b(nx, ny, h, eps, B, seed=100 + B)
    s = _solver(nx, ny, h, eps, prec)
    u, info = s.apply(b, sweeps=10, tol=1e-10, want_info=True)
    ref = O.solve(nx, ny, eps, b, route="band")
    assert O.rel_error_eq6(u.cpu().numpy(), ref) < 1e-6
    assert info.converged == 1 and info.rel_residual <= 1e-10


def test_refinement_contracts():
    """Each sweep shrinks the error (the stored inverse is a contraction
    preconditioner for this grid)."""
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_fourier(nx, ny, h, seed=1)
    b = _b(nx, ny, h, eps, 32, seed=5)
    ref = O.solve(nx, ny, eps, b, route="band")
    s = _solver(nx, ny, h, eps, "bf16")
    errs = [O.rel_error_eq6(s.apply(b, sweeps=k).cpu().numpy(), ref) for k in range(4)]
    assert errs[0] < 2e-2
    for a, c in zip(errs, errs[1:]):
        assert c < 0.5 * a, errs


def test_edge_cases():
    s = _solver(9, 8, 0.125, None, "bf16")
    empty = torch.empty((0, s.n), dtype=torch.float64, device="cuda")
    assert s.apply(empty).shape == (0, s.n)
    from paper_1602_00001_gb300.binding import PideError
    with pytest.raises(PideError):
        _solver(6, 6, 0.2, -np.ones((6, 6)), "bf16")
    b = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(PideError):
        s.apply(b, u=b)
    # zero right-hand side -> zero solution, in every path
    for B in (1, 20):
        z = torch.zeros((B, s.n), dtype=torch.float64, device="cuda")
        assert float(s.apply(z, sweeps=2).abs().max()) == 0.0


def test_apply_host_matches_device():
    nx = ny = 30
    h = 1.0 / 29
    eps = W.eps_lognormal(nx, ny, seed=9)
    b = _b(nx, ny, h, eps, 12, seed=3)
    s = _solver(nx, ny, h, eps, "bf16")
    ud = s.apply(b, sweeps=3).cpu().numpy()
    uh = s.apply_host(b, sweeps=3)
    # split (stream-K) tiles add FP64 partial sums atomically: order may differ
    assert np.max(np.abs(ud - uh)) <= 1e-14 * np.max(np.abs(ud))


def test_apply_host_pipelined_chunks():
    """B >= 512: host copies overlap the solves of two column chunks; same
    answer as the device apply (up to the chunked GEMM's FP32 rounding)."""
    nx = ny = 34
    h = 1.0 / 33
    eps = W.eps_lognormal(nx, ny, seed=19)
    b = _b(nx, ny, h, eps, 700, seed=4)
    s = _solver(nx, ny, h, eps, "bf16")
    ud = s.apply(b, sweeps=5).cpu().numpy()
    bh = torch.from_numpy(b).pin_memory()
    uh = torch.empty_like(bh).pin_memory()
    s.apply_host(bh, uh, sweeps=5)
    ref = O.solve(nx, ny, eps, b, route="band")
    assert O.rel_error_eq6(uh.numpy(), ref) < 1e-6
    assert np.max(np.abs(uh.numpy() - ud)) <= 1e-8 * np.max(np.abs(ud))


def test_save_load_roundtrip(tmp_path):
    nx, ny = 26, 21
    h = 1.0 / 25
    eps = W.eps_lognormal(nx, ny, seed=12)
    from paper_1602_00001_gb300.binding import Solver
    s = Solver(nx, ny, h, eps, "bf16")
    b = _b(nx, ny, h, eps, 20, seed=1)
    u1 = s.apply(b, sweeps=2).cpu().numpy()
    path = str(tmp_path / "inv.pide")
    s.save(path)
    s2 = Solver.load(path)
    u2 = s2.apply(b, sweeps=2).cpu().numpy()
    assert np.max(np.abs(u1 - u2)) <= 1e-14 * np.max(np.abs(u1))
    assert np.array_equal(s.inverse_row(7), s2.inverse_row(7))


@pytest.mark.parametrize("B", [64, 300])
def test_streamk_matches_whole_tiles(B):
    """The stream-K tail (k-block split, atomic partial sums) and whole-tile
    scheduling give the same contraction up to FP32 partial-sum rounding."""
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_lognormal(nx, ny, seed=21)
    b = _b(nx, ny, h, eps, B, seed=22)
    s = _solver(nx, ny, h, eps, "bf16")
    s.set_tuning(gemm_streamk=1)
    u1 = s.apply(b, sweeps=0).cpu().numpy()
    s.set_tuning(gemm_streamk=0)
    u0 = s.apply(b, sweeps=0).cpu().numpy()
    mag = s.apply(np.abs(b), sweeps=0).cpu().numpy()     # L^-1 >= 0: the |.| contraction
    assert np.all(np.abs(u1 - u0) <= 2e-5 * mag + 1e-300)


@pytest.mark.parametrize("prec", ["fp8x2", "fp8"])
@pytest.mark.parametrize("B", [16, 64, 300])
def test_fp8_single_apply_is_exact_contraction(prec, B):
    """kind::f8f6f4 GEMM: one apply equals the FP64 contraction of the
    oracle's own e4m3 rounding of the inverse (per-row scale, hi [+ lo]) and
    of the right-hand side (per-column scale), up to FP32 accumulation."""
    nx, ny = 40, 33
    h = 1.0 / 39
    eps = W.eps_fourier(nx, ny, h, seed=11)
    b = _b(nx, ny, h, eps, B, seed=B + 7)
    s = _solver(nx, ny, h, eps, prec)
    u = s.apply(b, sweeps=0).cpu().numpy()
    Linv = O.interior_inverse(nx, ny, eps)
    rs, hi, lo = O.quantize_rows_e4m3(Linv, prec == "fp8x2")
    Q = hi + lo
    t = O.round_fp32(np.max(np.abs(b), axis=1) / 448.0)
    isc = O.round_fp32(1.0 / t)
    r = O.round_e4m3(O.round_fp32(b * isc[:, None]))
    ref = (rs[:, None] * (Q @ r.T)).T * t[:, None]
    mag = (rs[:, None] * (np.abs(Q) @ np.abs(r).T)).T * t[:, None]
    err = np.abs(u - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))
    # the stored rows the library reports are scale * (hi + lo)
    row = s.inverse_row(3)
    assert np.max(np.abs(row - rs[3] * Q[3])) <= 1e-6 * np.max(np.abs(Q[3])) * rs[3]


@pytest.mark.parametrize("B", [1, 64, 300])
def test_fp8x2_refined_reaches_1e6(B):
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_fourier(nx, ny, h, seed=1)
    b = _b(nx, ny, h, eps, B, seed=300 + B)
    s = _solver(nx, ny, h, eps, "fp8x2")
    u = s.apply(b, sweeps=10)
    ref = O.solve(nx, ny, eps, b, route="band")
    assert O.rel_error_eq6(u.cpu().numpy(), ref) < 1e-6


def test_apply_in_cuda_graph():
    """The refined apply (prep, GEMM, residual sweeps) captured once in a CUDA
    graph and replayed gives the eager result."""
    nx = ny = 44
    h = 1.0 / 43
    eps = W.eps_lognormal(nx, ny, seed=31)
    b = torch.from_numpy(_b(nx, ny, h, eps, 96, seed=32)).cuda()
    s = _solver(nx, ny, h, eps, "bf16")
    s.set_tuning(gemm_streamk=0)          # whole tiles: bitwise-repeatable
    s.reserve(96)
    u_eager = s.apply(b, sweeps=4)
    u = torch.zeros_like(b)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        s.apply(b, u, sweeps=4, stream=st)          # warm-up outside capture
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        s.apply(b, u, sweeps=4, stream=st)
    u.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, u_eager)


@pytest.mark.parametrize("B", [512, 640])
def test_overlapped_refinement(B):
    """Residual of one column group on the aux stream under the other group's
    apply: same result as the single-stream schedule up to FP32 partial-sum
    rounding, reaches the oracle, and replays from a captured CUDA graph."""
    nx = ny = 48
    h = 1.0 / 47
    eps = W.eps_fourier(nx, ny, h, seed=41)
    b_np = _b(nx, ny, h, eps, B, seed=42)
    b = torch.from_numpy(b_np).cuda()
    s = _solver(nx, ny, h, eps, "bf16")
    s.reserve(B)
    s.set_tuning(overlap=0)
    u_seq = s.apply(b, sweeps=6)
    s.set_tuning(overlap=1)
    u_ovl = s.apply(b, sweeps=6)
    ref = O.solve(nx, ny, eps, b_np, route="band")
    assert O.rel_error_eq6(u_ovl.cpu().numpy(), ref) < 1e-6
    assert float((u_ovl - u_seq).abs().max()) <= 1e-8 * float(u_seq.abs().max())
    s.set_tuning(gemm_streamk=0)
    u_eager = s.apply(b, sweeps=6)
    u = torch.zeros_like(b)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        s.apply(b, u, sweeps=6, stream=st)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        s.apply(b, u, sweeps=6, stream=st)
    u.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, u_eager)


@pytest.mark.parametrize("nx,ny", [(40, 33), (131, 12), (12, 140), (3, 3)])
def test_symv_single_apply_is_exact_contraction(nx, ny):
    """B = 1 through the packed lower triangle of S^-1 = L^-1 D^-1 (BF16 hi +
    FP16 lo with a power-of-two scale per row, 128 x 128 tiles; upper blocks
    are the transposes of the stored lower ones) with x = D r formed in FP32:
    equals the FP64 contraction of the same rounded operands up to FP32
    accumulation."""
    h = 1.0 / (max(nx, ny) - 1)
    eps = W.eps_lognormal(nx, ny, seed=nx + ny)
    b = _b(nx, ny, h, eps, 1, seed=5)
    s = _solver(nx, ny, h, eps, "bf16")
    u = s.apply(b, sweeps=0).cpu().numpy()
    Linv = O.interior_inverse(nx, ny, eps)
    d = O.diagonal_d(nx, ny, eps)
    S = Linv / d[None, :]
    hi = O.round_bf16(S)
    sig = O.pow2_scale(np.max(np.abs(S - hi), axis=1), 15)
    Sl = hi + sig[:, None] * O.round_fp16((S - hi) / sig[:, None])
    blk = np.arange(s.n) // 128
    lower = blk[:, None] >= blk[None, :]
    A = np.where(lower, Sl, Sl.T)
    x = O.round_fp32(O.round_fp32(b[0]) * O.round_fp32(d))
    ref = A @ x
    mag = np.abs(A) @ np.abs(x)
    err = np.abs(u[0] - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))
    # two terms (~19 bits): one apply is already close to the exact solution
    assert O.rel_error_eq6(u, (Linv @ b[0])[None, :]) < 5e-6


def test_symv_one_apply_at_198sq():
    """198^2 unknowns: the symmetric two-term store alone (no refinement sweep),
    as the benchmark's B = 1 figure runs it (its operator: Fourier eps seed 5,
    moving charges seed 5), within 5e-7 of the FP64 GPU apply on three
    right-hand sides and within 1e-6 of the oracle on two of them."""
    nx = ny = 200
    h = 1.0 / 199
    eps = W.eps_fourier(nx, ny, h, seed=5)
    rho = W.moving_charges(nx, ny, h, seed=5, steps=3)
    s = _solver(nx, ny, h, eps, "fp16_fp8")
    b = s.rhs_from_charge(torch.from_numpy(rho).cuda())
    u = torch.stack([s.apply(b[k:k + 1], sweeps=0)[0] for k in range(3)])
    s.close()
    s64 = _solver(nx, ny, h, eps, "fp64")
    u64 = s64.apply(b)
    d = ((u - u64).abs().amax(dim=1) / u64.abs().amax(dim=1)).max().item()
    assert d < 5e-7, d
    ref = O.solve(nx, ny, eps, b[:2].cpu().numpy(), route="band")
    assert O.rel_error_eq6(u[:2].cpu().numpy(), ref) < 1e-6


def test_symv_refined_matches_gemv():
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_fourier(nx, ny, h, seed=8)
    b = _b(nx, ny, h, eps, 1, seed=9)
    ref = O.solve(nx, ny, eps, b, route="band")
    s = _solver(nx, ny, h, eps, "bf16")
    for symv in (1, 0):
        s.set_tuning(symv=symv)
        u = s.apply(b, sweeps=6).cpu().numpy()
        assert O.rel_error_eq6(u, ref) < 1e-6, symv
