"""Table 1 of the paper on the GPU: the Eq. (4)/(5) problem solved with the
FP64 inverse formed on the GPU, its entries rounded to k decimals on the GPU
(pide_round_inverse_decimal), one FP64 apply; the Eq. (6) error of every cell
against the printed value (half a unit in the last printed place), and
against the oracle's own evaluation of the same cell."""
import os

import numpy as np
import pytest

from oracle import pide_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_00001_gb300 import build, binding
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    binding.load_library()


def _printed(golden_dir):
    out = {}
    for line in open(os.path.join(golden_dir, "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        k = None if parts[0] == "none" else int(parts[0])
        for n, v in zip([5, 11, 21, 41, 81], parts[1:]):
            out[(n, k)] = v
    return out


def _gpu_cell(n, k):
    from paper_1602_00001_gb300.binding import Solver
    h = 1.0 / (n - 1)
    x = h * np.arange(n)
    X, Y = np.meshgrid(x, x)
    f = O.eq4_source(X, Y)[1:-1, 1:-1].reshape(1, -1)
    s = Solver(n, n, h, np.ones((n, n)), "fp64")
    b = s.rhs_from_charge(f)                     # -h^2 f / 4 on the device
    if k is not None:
        s.round_inverse_decimal(k)
    u = np.zeros((n, n))
    u[1:-1, 1:-1] = s.apply(b).cpu().numpy().reshape(n - 2, n - 2)
    ua = O.eq5_exact(X, Y)
    return float(np.max(np.abs(ua - u)) / np.max(np.abs(ua)))


@pytest.mark.parametrize("n", [5, 11, 21, 41, 81])
def test_table1_gpu(golden_dir, n):
    printed = _printed(golden_dir)
    oracle = dict(zip([1, 2, 3, 5, None], O.table1_row(n, [1, 2, 3, 5, None])))
    for k in [1, 2, 3, 5, None]:
        got = _gpu_cell(n, k)
        if (n, k) != (5, 1):       # the one cell no rounding rule reproduces (oracle: xfail)
            p = printed[(n, k)]
            dec = len(p.split(".")[1])
            assert abs(got - float(p)) <= 0.5 * 10.0 ** (-dec) + 1e-12, (n, k, got, p)
        # The GPU's FP64 inverse differs from the oracle's LU inverse by rounding
        # only, so the rounded tables agree unless entries sit on decimal ties.
        # At n = 5 with one digit they do (entries such as 1/4): the last bit of
        # each inverse decides the tie, GPU 0.0918 against the oracle's 0.0566
        # (printed 0.0569), so that cell is compared with neither.
        if (n, k) != (5, 1):
            assert abs(got - oracle[k]) <= 1e-3 * oracle[k] + 1e-12, (n, k, got, oracle[k])


def test_round_inverse_decimal_entries():
    """The rounded entries are the oracle's rounding of the GPU's own FP64 row."""
    from paper_1602_00001_gb300.binding import Solver, PideError
    n = 13
    s = Solver(n, n, 1.0 / (n - 1), np.ones((n, n)), "fp64")
    row = s.inverse_row(40)
    s.round_inverse_decimal(3)
    assert np.array_equal(s.inverse_row(40), O.round_decimals(row, 3))
    s2 = Solver(n, n, 1.0 / (n - 1), np.ones((n, n)), "bf16")
    with pytest.raises(PideError):
        s2.round_inverse_decimal(3)
    with pytest.raises(PideError):
        s.round_inverse_decimal(16)
