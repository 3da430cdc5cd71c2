"""The refinement's measured contraction: reported per call in pide_info, and
deciding the stored format per grid in pide_setup_auto (the binary analogue
of the paper's rounding study, Table 1: the inverse rounded to each candidate
format, the error of the refined apply measured for each).

* pide_info.contraction equals (||r_K|| / ||r_0||)^(1/K) computed from FP64
  residuals of separate solves with 0 and K sweeps; NaN without a sweep;
  pide_info.ms is the call's device time.
* pide_setup_auto on the moving-charge workload at 21^2, 81^2 and 198^2
  unknowns keeps a 16-bit store with one sweep (the formats study of the
  design notes: FP16 + e4m3 or FP16 reach the target in one sweep, BF16 needs
  two or more), and PIDE_SWEEPS_AUTO then reaches 1e-6 against the oracle.
* With its built-in probes (no probe given) the choice also serves the
  workload to 1e-6."""
import math

import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_00001_gb300 import build, binding
    build.build()
    binding.load_library()


def _rel_residual(s, b, u):
    r = s.residual(b, u)
    return float((r.abs().amax(dim=1) / b.abs().amax(dim=1)).max())


@pytest.mark.parametrize("prec,sweeps", [("bf16", 3), ("fp16", 2), ("fp16_fp8", 1),
                                         ("fp64", 1)])
def test_info_contraction_matches_fp64_residuals(prec, sweeps):
    from paper_1602_00001_gb300.binding import Solver
    nx = ny = 60
    h = 1.0 / 59
    eps = W.eps_fourier(nx, ny, h, seed=3)
    s = Solver(nx, ny, h, eps, prec)
    # whole tiles only: the stream-K tail adds FP32 partial sums with FP64
    # atomics in a varying order, and the solves compared here must match
    s.set_tuning(gemm_streamk=0)
    b = s.rhs_from_charge(torch.from_numpy(W.moving_charges(nx, ny, h, seed=2, steps=200)).cuda())
    u0 = s.apply(b, sweeps=0)
    uk, info = s.apply(b, sweeps=sweeps, want_info=True)
    r0, rk = _rel_residual(s, b, u0), _rel_residual(s, b, uk)
    assert info.sweeps == sweeps and info.converged == 1
    assert abs(info.rel_residual - rk) <= 1e-9 * rk + 1e-300
    expect = (rk / r0) ** (1.0 / sweeps)
    assert abs(info.contraction - expect) <= 1e-6 * expect, (info.contraction, expect)
    if prec != "fp64":
        assert 0.0 < info.contraction < 0.5
    assert info.ms > 0.0
    _, info0 = s.apply(b, sweeps=0, want_info=True)
    assert math.isnan(info0.contraction) and info0.ms > 0.0
    s.close()


def test_info_contraction_with_tolerance():
    """A tolerance-driven solve reports the contraction over the sweeps it ran."""
    from paper_1602_00001_gb300.binding import Solver
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_lognormal(nx, ny, seed=5)
    s = Solver(nx, ny, h, eps, "bf16")
    s.set_tuning(gemm_streamk=0)
    b = s.rhs_from_charge(torch.from_numpy(W.gaussian_blobs(nx, ny, h, 3, batch=40)).cuda())
    u, info = s.apply(b, sweeps=12, tol=1e-9, want_info=True)
    assert info.converged == 1 and 1 <= info.sweeps < 12
    u0 = s.apply(b, sweeps=0)
    r0 = _rel_residual(s, b, u0)
    expect = (info.rel_residual / r0) ** (1.0 / info.sweeps)
    assert abs(info.contraction - expect) <= 1e-6 * expect
    s.close()


def _workload(nodes, cols=16):
    h = 1.0 / (nodes - 1)
    eps = W.eps_fourier(nodes, nodes, h, seed=5)
    steps = 1024
    rho = W.moving_charges(nodes, nodes, h, seed=5, steps=steps)
    pick = list(range(0, steps, steps // cols))[:cols]
    b = O.rhs_from_charge(nodes, nodes, h, eps, rho[pick])
    return h, eps, b


@pytest.mark.parametrize("nodes", [23, 83, 200])
def test_auto_chooses_a_one_sweep_16bit_store(nodes):
    from paper_1602_00001_gb300.binding import SWEEPS_AUTO, Solver
    h, eps, b = _workload(nodes)
    s = Solver.auto(nodes, nodes, h, eps, target=0.5e-6, probe=b)
    rep = s.auto_report()
    names = [c["precision"] for c in rep["candidates"]]
    assert names[:4] == ["fp16_fp8", "fp16", "bf16_fp8", "bf16"]
    assert rep["chosen"] in ("fp16_fp8", "fp16") and rep["sweeps"] == 1, rep
    assert s.precision == rep["chosen"] and s.info().sweeps_hint == 1
    bf16 = rep["candidates"][3]
    assert bf16["sweeps"] >= 2 and bf16["contraction"] > rep["candidates"][1]["contraction"]
    chosen = [c for c in rep["candidates"] if c["precision"] == rep["chosen"]][0]
    assert chosen["error"] <= 0.5e-6
    assert chosen["cost"] == min(c["cost"] for c in rep["candidates"] if c["sweeps"] >= 0)
    # the chosen store with its measured sweep count, against the oracle
    u = s.apply(torch.from_numpy(b).cuda(), sweeps=SWEEPS_AUTO).cpu().numpy()
    cols = [0, 15] if nodes == 200 else list(range(16))
    ref = O.solve(nodes, nodes, eps, b[cols], route="band")
    assert O.rel_error_eq6(u[cols], ref) < 1e-6
    s.close()


def test_auto_builtin_probe_serves_the_workload():
    from paper_1602_00001_gb300.binding import SWEEPS_AUTO, Solver
    nodes = 83
    h, eps, b = _workload(nodes)
    s = Solver(nodes, nodes, h, eps, "auto")
    rep = s.auto_report()
    assert rep["nprobe"] == 16 and rep["target"] == 0.5e-6
    assert s.precision == rep["chosen"] and rep["sweeps"] >= 0
    u = s.apply(torch.from_numpy(b).cuda(), sweeps=SWEEPS_AUTO).cpu().numpy()
    ref = O.solve(nodes, nodes, eps, b, route="band")
    assert O.rel_error_eq6(u, ref) < 1e-6
    s.close()


def test_sweeps_auto_needs_an_auto_handle():
    from paper_1602_00001_gb300.binding import PideError, SWEEPS_AUTO, Solver
    s = Solver(20, 20, 1.0 / 19, None, "bf16")
    assert s.info().sweeps_hint == -1
    with pytest.raises(PideError):
        s.apply(np.zeros((2, s.n)), sweeps=SWEEPS_AUTO)
    with pytest.raises(PideError):
        s.auto_report()
    s.close()


def test_auto_3d():
    """PIDE_AUTO on a 3-D grid (pide_setup_3d): the chosen store with its
    measured sweep count reaches the 3-D oracle to 1e-6."""
    from oracle import pide_oracle3d as O3
    from paper_1602_00001_gb300.binding import SWEEPS_AUTO, Solver3D
    nx, ny, nz = 14, 13, 12
    rng = np.random.default_rng(8)
    eps = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    n = (nx - 2) * (ny - 2) * (nz - 2)
    b = rng.standard_normal((40, n))
    s = Solver3D(nx, ny, nz, 1.0 / (nx - 1), eps, "auto")
    rep = s.auto_report()
    assert s.precision == rep["chosen"] and rep["sweeps"] >= 0
    u = s.apply(b, sweeps=SWEEPS_AUTO).cpu().numpy()
    ref = O3.solve(nx, ny, nz, eps, b[[0, 39]], route="band")
    assert np.max(np.abs(u[[0, 39]] - ref)) / np.max(np.abs(ref)) < 1e-6
    s.close()
