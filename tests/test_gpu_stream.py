"""GPU parity of the time-stepping driver pide_solve_stream: a sequence of
right-hand sides (or charge densities) in host memory, solved in chunks with
the copies overlapping the solves, equals the device apply of each chunk and
the oracle's solution."""
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


def _setup(T, seed):
    nx = ny = 50
    h = 1.0 / 49
    eps = W.eps_fourier(nx, ny, h, seed=seed)
    rho = W.moving_charges(nx, ny, h, seed=seed + 1, steps=T)
    return nx, ny, h, eps, rho


@pytest.mark.parametrize("T,chunk", [(2500, 1024), (700, 1024), (5, 2), (3, 1)])
def test_stream_equals_chunked_device_apply(T, chunk):
    """Ragged last chunk, a single chunk, odd chunks, one column per chunk.
    The driver cuts the sequence into its own pieces (a half chunk first
    and last), so a column may go through another apply kernel than in a
    device apply of `chunk` columns: the two refined results agree to the
    refinement's accuracy, and both to the oracle's."""
    nx, ny, h, eps, rho = _setup(T, 40)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    s = _solver(nx, ny, h, eps, "bf16")
    u = s.solve_stream(b, chunk=chunk, sweeps=4)
    for c0 in range(0, T, chunk):
        ud = s.apply(b[c0:c0 + chunk], sweeps=4).cpu().numpy()
        d = np.abs(u[c0:c0 + chunk] - ud).max(axis=1) / np.abs(ud).max(axis=1)
        assert d.max() <= 1e-7, (c0, float(d.max()))
    cols = [0, T // 2, T - 1]
    ref = O.solve(nx, ny, eps, b[cols], route="band")
    assert O.rel_error_eq6(u[cols], ref) < 1e-6


def test_stream_from_charge_pinned():
    """charge = 1: b = -h^2 rho / d formed on the device; pinned torch buffers."""
    T = 1500
    nx, ny, h, eps, rho = _setup(T, 41)
    s = _solver(nx, ny, h, eps, "bf16")
    rho_t = torch.from_numpy(rho).pin_memory()
    u_t = torch.empty_like(rho_t).pin_memory()
    s.solve_stream(rho_t, u_t, chunk=512, sweeps=4, charge=True)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    cols = [0, 511, 512, 1499]
    ref = O.solve(nx, ny, eps, b[cols], route="band")
    assert O.rel_error_eq6(u_t.numpy()[cols], ref) < 1e-6
    # the input buffer is not modified (the conversion runs on the device copy)
    assert np.array_equal(rho_t.numpy(), rho)


def test_stream_fp64_and_arguments():
    from paper_1602_00001_gb300.binding import PideError
    T = 40
    nx, ny, h, eps, rho = _setup(T, 42)
    b = O.rhs_from_charge(nx, ny, h, eps, rho)
    s = _solver(nx, ny, h, eps, "fp64")
    u = s.solve_stream(b, chunk=16)
    ref = O.solve(nx, ny, eps, b, route="band")
    assert O.rel_error_eq6(u, ref) < 1e-12
    s.solve_stream(np.zeros((0, s.n)))                     # T = 0: nothing to do
    with pytest.raises(PideError):
        s.solve_stream(b, chunk=0)
    with pytest.raises(PideError):
        s.solve_stream(b, b)                                # in == u
