"""The SM-pair tensor-core apply with its last round of tiles cut along K.

The tiles of the last partial round of 256 x 256 tiles are split into
K-ranges whose FP32 partial tiles a reduction kernel adds to u in FP64.  The
default weighs the reduction's cost and does not split at these small sizes;
the tests take gemm_streamk = 2, which leaves that cost out.  On a 60 x 60 node
grid (n = 3364, 14 row slabs of 256; 53 k-blocks of 64, 27 of
128 for the e4m3 correction) with 76 pairs: B = 300 gives 28 tiles (no whole
round, every tile in 5 pieces), B = 1600 gives 98 tiles (one whole round, then
22 tiles in 3 pieces), B = 1024 gives 56 tiles in 4 pieces (three pieces on
most pairs; the correction GEMM's 27 k-blocks allow no gain: whole tiles),
B = 1200 gives 70 tiles (no split: the last round is nearly full).  Each
result is checked against the oracle's exact contraction of the same rounded
operands (the bound of the FP32 accumulation), against the whole-tile schedule,
for determinism, and through the profile's 'reduce' class.
"""
import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX = NY = 60
H = 1.0 / 59


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_00001_gb300 import build, binding
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    binding.load_library()


@pytest.fixture(scope="module")
def eps():
    return W.eps_lognormal(NX, NY, seed=41)


@pytest.fixture(scope="module")
def linv(eps):
    return O.interior_inverse(NX, NY, eps)


def _b(eps, B, seed):
    rho = W.gaussian_blobs(NX, NY, H, seed, batch=B)
    return O.rhs_from_charge(NX, NY, H, eps, rho)


def _solver(eps, prec, streamk=2):
    from paper_1602_00001_gb300.binding import Solver
    s = Solver(NX, NY, H, eps, prec)
    s.set_tuning(gemm_streamk=streamk)
    return s


def _expected(linv, b, prec):
    """The first apply's exact value from the oracle's roundings, and the
    contraction of magnitudes that bounds its FP32 accumulation error."""
    if prec == "bf16":
        Q = O.round_bf16(linv)
        R = O.round_bf16(b)
        return (Q @ R.T).T, (np.abs(Q) @ np.abs(R).T).T
    sc, Q, cc, C = O.quantize_fp16_correction(linv)
    t, R = O.quantize_cols_fp16(b)
    ref = (sc[:, None] * (Q @ R.T)).T * t[:, None]
    mag = (sc[:, None] * (np.abs(Q) @ np.abs(R).T)).T * t[:, None]
    if prec == "fp16_fp8":
        tc = O.round_fp32(np.max(np.abs(R), axis=1) / 448.0)
        tc = np.where(tc > 0, tc, 1.0)
        r8 = O.round_e4m3(O.round_fp32(R * O.round_fp32(1.0 / tc)[:, None]))
        ref = ref + (cc[:, None] * (C @ r8.T)).T * (tc * t)[:, None]
        mag = mag + (cc[:, None] * (np.abs(C) @ np.abs(r8).T)).T * (tc * t)[:, None]
    return ref, mag


def _accumulation_bound(n):
    """FP32 accumulation bound relative to the contraction of magnitudes: the
    tensor core adds each K = 16 step of the 16-bit GEMM (4 per 64-element
    k-block) to its FP32 accumulator with an error near one ulp (2^-23) of the
    running sum; L^-1 >= 0 and the blob right-hand sides keep the sums growing
    in one direction, so the errors can add up linearly.  Two ulps per step."""
    steps = 4 * ((n + 63) // 64)
    return 2.0 * steps * 2.0 ** -23


# reduction launches of one unrefined apply: (FP16 / BF16 GEMM, e4m3 correction GEMM)
REDUCES = {300: (1, 1), 1600: (1, 1), 1024: (1, 0), 1200: (0, 0)}


@pytest.mark.parametrize("B", [300, 1600, 1024, 1200])
@pytest.mark.parametrize("prec", ["fp16", "fp16_fp8", "bf16"])
def test_first_apply_is_exact_contraction(eps, linv, prec, B):
    b = _b(eps, B, seed=B + 7)
    b[B // 2] *= 1e-20                     # a column far below the others' scale
    s = _solver(eps, prec)
    with s.profile() as prof:
        u = s.apply(b, sweeps=0).cpu().numpy()
    ref, mag = _expected(linv, b, prec)
    ratio = np.abs(u - ref) / (mag + 1e-300)
    j, p = np.unravel_index(np.argmax(ratio), ratio.shape)
    tile = (p // 256) * ((B + 255) // 256) + j // 256
    assert ratio.max() <= _accumulation_bound(s.n), (float(ratio.max()), int(p), int(j), int(tile))
    main, corr = REDUCES[B]
    assert prof["reduce"][0] == main + (corr if prec == "fp16_fp8" else 0), prof
    s.close()


@pytest.mark.parametrize("B", [1600, 1024])
@pytest.mark.parametrize("prec", ["fp16_fp8", "bf16"])
def test_split_matches_whole_tiles_and_repeats(eps, prec, B):
    """Same contraction as whole tiles up to FP32 partial-sum rounding (bounded by
    the magnitudes, L^-1 >= 0); two runs of the split schedule are identical."""
    b = _b(eps, B, seed=5)
    s = _solver(eps, prec)
    bd = torch.from_numpy(b).cuda()
    u1 = s.apply(bd, sweeps=1)
    u2 = s.apply(bd, sweeps=1)
    assert torch.equal(u1, u2)
    s.set_tuning(gemm_streamk=0)
    with s.profile() as prof:
        u0 = s.apply(bd, sweeps=1)
    assert prof["reduce"][0] == 0
    mag = s.apply(bd.abs(), sweeps=0)
    assert bool(((u1 - u0).abs() <= 1e-4 * mag + 1e-300).all())
    s.close()


def test_refined_split_reaches_oracle(eps, linv):
    """One refinement sweep through split applies (the sweep accumulates into u
    in the reduction) reaches the FP64 oracle to 1e-6."""
    B = 1600
    b = _b(eps, B, seed=9)
    s = _solver(eps, "fp16_fp8")
    with s.profile() as prof:
        u = s.apply(b, sweeps=1).cpu().numpy()
    assert prof["reduce"][0] == 3, prof      # first apply, its correction term, the sweep
    cols = [0, 799, 1599]
    ref = (linv @ b[cols].T).T
    assert O.rel_error_eq6(u[cols], ref) < 1e-6


def test_converged_tolerance_skips_the_reduction(eps):
    """With a tolerance met after the first apply, the later applies and their
    reductions return early: u equals the unrefined result (a reduction that
    ran anyway would add the previous GEMM's partial tiles)."""
    B = 1600
    b = torch.from_numpy(_b(eps, B, seed=11)).cuda()
    s = _solver(eps, "fp16")
    u0 = s.apply(b, sweeps=0)
    ut = s.apply(b, sweeps=3, tol=1e-2)
    mag = u0.abs().amax()
    assert float((ut - u0).abs().max() / mag) <= 1e-12
    s.close()


def test_tiny_grid_keeps_whole_tiles():
    """Too few k-blocks for pieces of 8 (n = 361: 6 blocks of 64): whole tiles."""
    nx = ny = 21
    h = 1.0 / 20
    e = W.eps_lognormal(nx, ny, seed=3)
    rho = W.gaussian_blobs(nx, ny, h, 4, batch=300)
    b = O.rhs_from_charge(nx, ny, h, e, rho)
    from paper_1602_00001_gb300.binding import Solver
    s = Solver(nx, ny, h, e, "bf16")
    s.set_tuning(gemm_streamk=2)
    with s.profile() as prof:
        u = s.apply(b, sweeps=4).cpu().numpy()
    assert prof["reduce"][0] == 0
    ref = (O.interior_inverse(nx, ny, e) @ b.T).T
    assert O.rel_error_eq6(u, ref) < 1e-6
    s.close()


def test_default_weighs_the_reduction(eps):
    """The default (gemm_streamk = 1) counts each partial tile's reduction as
    half a k-block: at 53 k-blocks per tile the 28 tiles of B = 300 stay whole
    (140 partial tiles would cost more than the 0.6 of a tile they save), while
    gemm_streamk = 2 splits them; both equal the oracle's contraction."""
    B = 300
    b = _b(eps, B, seed=13)
    res = {}
    for sk in (1, 2):
        s = _solver(eps, "fp16", streamk=sk)
        with s.profile() as prof:
            res[sk] = s.apply(b, sweeps=0)
        assert prof["reduce"][0] == (0 if sk == 1 else 1), (sk, prof)
        if sk == 2:
            mag = s.apply(np.abs(b), sweeps=0)     # L^-1 >= 0: the contraction of |b|
        s.close()
    assert bool(((res[1] - res[2]).abs() <= 1e-4 * mag + 1e-300).all())


def test_split_apply_in_cuda_graph(eps):
    """The refined apply with K-split GEMMs and their reductions, captured once
    in a CUDA graph and replayed twice, gives the eager result bit for bit (the
    reduction adds the partials in a fixed order)."""
    B = 1600
    b = torch.from_numpy(_b(eps, B, seed=21)).cuda()
    s = _solver(eps, "fp16_fp8")
    s.reserve(B)
    u_eager = s.apply(b, sweeps=1)
    u = torch.zeros_like(b)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        s.apply(b, u, sweeps=1, stream=st)          # warm-up outside capture
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        s.apply(b, u, sweeps=1, stream=st)
    for _ in range(2):
        u.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(u, u_eager)
    s.close()


def test_split_3d_reaches_oracle():
    """The 3-D operator through split GEMMs: 18 x 18 x 18 nodes (4096 unknowns,
    16 row slabs, 64 k-blocks), B = 300 (32 tiles of the last round, all
    split), FP16 + e4m3 with one sweep, against the 3-D oracle."""
    from oracle import pide_oracle3d as O3
    from paper_1602_00001_gb300.binding import Solver3D
    nx = ny = nz = 18
    rng = np.random.default_rng(5)
    e3 = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    b = rng.standard_normal((300, 16 ** 3))
    s = Solver3D(nx, ny, nz, 1.0 / (nx - 1), e3, "fp16_fp8")
    s.set_tuning(gemm_streamk=2)
    with s.profile() as prof:
        u = s.apply(b, sweeps=1).cpu().numpy()
    assert prof["reduce"][0] >= 2, prof          # the FP16 applies (and the correction GEMM's)
    cols = [0, 150, 299]
    ref = O3.solve(nx, ny, nz, e3, b[cols], route="band")
    assert O.rel_error_eq6(u[cols], ref) < 1e-6
    s.close()
