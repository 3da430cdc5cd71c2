"""GPU parity of the tensor-core apply on SM pairs (tcgen05 cta_group::2,
256 x 256 tiles; PIDE_TUNE_GEMM_2CTA): one apply equals the FP64 contraction
of the oracle's own roundings of the inverse and the right-hand side up to
FP32 accumulation, with and without the stream-K tail, in BF16 and FP8 hi+lo;
refined results equal the single-SM kernel's; a full-size launch on sampled
columns."""
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


@pytest.mark.parametrize("B", [129, 256, 300, 777])
@pytest.mark.parametrize("streamk", [0, 1])
def test_pair_bf16_single_apply_is_exact_contraction(B, streamk):
    nx, ny = 40, 33                     # n = 1178: five 256-row tiles, the last ragged
    h = 1.0 / 39
    eps = W.eps_fourier(nx, ny, h, seed=11)
    b = _b(nx, ny, h, eps, B, seed=B + 50)
    s = _solver(nx, ny, h, eps, "bf16")
    s.set_tuning(gemm_2cta=1, gemm_streamk=streamk)
    u = s.apply(b, sweeps=0).cpu().numpy()
    Q = O.round_bf16(O.interior_inverse(nx, ny, eps))
    f = O.round_bf16(b)
    ref, mag = (Q @ f.T).T, (np.abs(Q) @ np.abs(f).T).T
    err = np.abs(u - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))


@pytest.mark.parametrize("B", [200, 300])
def test_pair_fp8x2_single_apply_is_exact_contraction(B):
    nx, ny = 40, 33
    h = 1.0 / 39
    eps = W.eps_fourier(nx, ny, h, seed=11)
    b = _b(nx, ny, h, eps, B, seed=B + 7)
    s = _solver(nx, ny, h, eps, "fp8x2")
    s.set_tuning(gemm_2cta=1)
    u = s.apply(b, sweeps=0).cpu().numpy()
    Linv = O.interior_inverse(nx, ny, eps)
    rs, hi, lo = O.quantize_rows_e4m3(Linv, True)
    Q = hi + lo
    t = O.round_fp32(np.max(np.abs(b), axis=1) / 448.0)
    isc = O.round_fp32(1.0 / t)
    r = O.round_e4m3(O.round_fp32(b * isc[:, None]))
    ref = (rs[:, None] * (Q @ r.T)).T * t[:, None]
    mag = (rs[:, None] * (np.abs(Q) @ np.abs(r).T)).T * t[:, None]
    err = np.abs(u - ref)
    assert np.all(err <= 2e-5 * mag + 1e-300), float(np.max(err / mag))


def test_pair_refined_equals_single_sm():
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_lognormal(nx, ny, seed=12)
    b = _b(nx, ny, h, eps, 640, seed=13)
    s = _solver(nx, ny, h, eps, "bf16")
    assert s.get_tuning()["gemm_2cta"] == 1           # the default
    s.set_tuning(gemm_2cta=0)
    u1 = s.apply(b, sweeps=4).cpu().numpy()
    s.set_tuning(gemm_2cta=1)
    u2 = s.apply(b, sweeps=4).cpu().numpy()
    assert O.rel_error_eq6(u2, u1) < 1e-7
    ref = O.solve(nx, ny, eps, b[:3], route="band")
    assert O.rel_error_eq6(u2[:3], ref) < 1e-6


def test_pair_full_size_sampled():
    """198^2 unknowns, B = 1024, the bench's launch: sampled columns against
    the FP64 GPU apply (the refined result) and the single-SM kernel."""
    nx = ny = 200
    h = 1.0 / 199
    eps = W.eps_fourier(nx, ny, h, seed=1)
    rho = W.moving_charges(nx, ny, h, seed=5, steps=1024)
    s = _solver(nx, ny, h, eps, "bf16")
    b = s.rhs_from_charge(torch.from_numpy(rho).cuda())
    s.set_tuning(gemm_2cta=0)
    u1 = s.apply(b, sweeps=4)
    s.set_tuning(gemm_2cta=1)
    u2 = s.apply(b, sweeps=4)
    cols = [0, 255, 256, 511, 700, 1023]
    d = ((u2[cols] - u1[cols]).abs().amax(dim=1) / u1[cols].abs().amax(dim=1)).max().item()
    assert d < 1e-7, d
    b_np = b[cols[:2]].cpu().numpy()
    ref = O.solve(nx, ny, eps, b_np, route="band")
    assert O.rel_error_eq6(u2[cols[:2]].cpu().numpy(), ref) < 1e-6


def test_pair_stream_k_at_full_size():
    """198^2 unknowns, B = 256: 154 pair tiles on the resident pairs (about two
    waves), where the pair kernel takes the stream-K tail; against whole tiles."""
    nx = ny = 200
    h = 1.0 / 199
    eps = W.eps_fourier(nx, ny, h, seed=1)
    rho = W.moving_charges(nx, ny, h, seed=6, steps=256)
    s = _solver(nx, ny, h, eps, "bf16")
    b = s.rhs_from_charge(torch.from_numpy(rho).cuda())
    s.set_tuning(gemm_streamk=1)
    u1 = s.apply(b, sweeps=0)
    s.set_tuning(gemm_streamk=0)
    u0 = s.apply(b, sweeps=0)
    # the same FP32 sums in another order: bounded by the contraction of |Q| |R|
    d = ((u1 - u0).abs().amax(dim=1) / u0.abs().amax(dim=1)).max().item()
    assert d < 1e-4, d
