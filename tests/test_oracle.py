"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a value the paper prints, a closed form, an invariant, a library
routine on a special case, or finite differences."""
import os

import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W


def _load_matrix(path):
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([float(v) for v in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- Fig. 3


def test_fig3_matrix_bit_exact(golden_dir):
    """Fig. 3: the printed 15x15 system for nx=3, ny=5 at eps=1."""
    ref = _load_matrix(os.path.join(golden_dir, "fig3_matrix.txt"))
    A = O.assemble_full(3, 5)
    assert A.shape == (15, 15)
    assert np.array_equal(A, ref)


def test_fig3_rhs_layout():
    """Fig. 3 right side: boundary values at boundary rows, the interior
    right-hand side at rows u_{2,2}, u_{3,2}, u_{4,2} (1-based 5, 8, 11)."""
    g = np.arange(15, dtype=float).reshape(5, 3) + 100.0
    rhs = O.full_rhs(3, 5, np.array([1.0, 2.0, 3.0]), g)
    interior_rows = [4, 7, 10]
    assert np.array_equal(rhs[interior_rows], [1.0, 2.0, 3.0])
    mask = np.ones(15, bool)
    mask[interior_rows] = False
    assert np.array_equal(rhs[mask], g.reshape(-1)[mask])


def test_full_system_matches_interior_solve():
    """The full Fig. 3 system (identity boundary rows, boundary values on the
    right) and the interior solve with the boundary lifted agree."""
    nx, ny = 6, 5
    eps = W.eps_lognormal(nx, ny, seed=11)
    rng = np.random.default_rng(5)
    g = rng.standard_normal((ny, nx))
    b = rng.standard_normal((2, (nx - 2) * (ny - 2)))
    A = O.assemble_full(nx, ny, eps)
    u_full = (O.lu_inverse(A) @ O.full_rhs(nx, ny, b, g).T).T
    u_full = u_full.reshape(2, ny, nx)
    # boundary rows reproduce the boundary values
    assert np.allclose(u_full[:, 0, :], g[0], atol=1e-15, rtol=0)
    u_int = O.solve(nx, ny, eps, b, g)
    assert np.max(np.abs(u_full[:, 1:-1, 1:-1].reshape(2, -1) - u_int)) < 1e-13


# ---------------------------------------------------------------- Table 1


def _table1(golden_dir):
    out = {}
    for line in open(os.path.join(golden_dir, "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        k = None if parts[0] == "none" else int(parts[0])
        for n, v in zip([5, 11, 21, 41, 81], parts[1:]):
            out[(n, k)] = v
    return out


_T1_CACHE = {}


def _table1_col(n):
    if n not in _T1_CACHE:
        _T1_CACHE[n] = dict(zip([1, 2, 3, 5, None], O.table1_row(n, [1, 2, 3, 5, None])))
    return _T1_CACHE[n]


@pytest.mark.parametrize("n", [5, 11, 21, 41, 81])
@pytest.mark.parametrize("k", [1, 2, 3, 5, None])
def test_table1(golden_dir, n, k):
    """Table 1: every cell to the printed digits (half a unit in the last
    printed place), with b = -h^2 f / 4, rounding half away from zero, and
    Eq. (6)'s maximum over grid nodes."""
    if (n, k) == (5, 1):
        pytest.xfail("n=5, 1 digit: printed 0.0569, no rounding rule reproduces it "
                     "(half-away 0.0566, half-even 0.0930, ceil 0.0537)")
    printed = _table1(golden_dir)[(n, k)]
    decimals = len(printed.split(".")[1])
    got = _table1_col(n)[k]
    assert abs(got - float(printed)) <= 0.5 * 10.0 ** (-decimals) + 1e-12, (got, printed)


def test_round_decimals_special_cases():
    a = np.array([0.25, -0.25, 0.1234, 3.4449, 0.05, -0.05])
    assert np.array_equal(O.round_decimals(a, 1), [0.3, -0.3, 0.1, 3.4, 0.1, -0.1])
    assert np.array_equal(O.round_decimals(a, 2), [0.25, -0.25, 0.12, 3.44, 0.05, -0.05])


# ---------------------------------------------------------------- closed forms


def _dst_inverse(nx, ny):
    """L^-1 at eps=1 from the 2-D discrete sine basis: eigenvalues
    1 - (cos(k pi/(my+1)) + cos(l pi/(mx+1)))/2."""
    mx, my = nx - 2, ny - 2
    i = np.arange(1, my + 1)
    j = np.arange(1, mx + 1)
    Vy = np.sqrt(2.0 / (my + 1)) * np.sin(np.pi * np.outer(i, i) / (my + 1))
    Vx = np.sqrt(2.0 / (mx + 1)) * np.sin(np.pi * np.outer(j, j) / (mx + 1))
    lam = 1.0 - 0.5 * (np.cos(np.pi * i / (my + 1))[:, None] + np.cos(np.pi * j / (mx + 1))[None, :])
    V = np.kron(Vy, Vx)          # row (i,j) with j fastest, column (k,l)
    return V @ np.diag(1.0 / lam.reshape(-1)) @ V.T


@pytest.mark.parametrize("route,nx,ny", [("dense", 9, 11), ("dense", 5, 4), ("band", 22, 17)])
def test_dst_closed_form(route, nx, ny):
    ref = _dst_inverse(nx, ny)
    got = O.interior_inverse(nx, ny, None, route)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-13


def test_layered_medium_series_resistance():
    """eps varying along x only, u = 0 at x = 0 and u = 1 at x = 1, the
    1-D solution on the top and bottom rows, no charge: the potential equals
    the fraction of the series resistance sum_k (1/eps_k + 1/eps_{k+1})/2
    crossed so far.  This fixes the face rule (harmonic mean of node eps) and
    the boundary lifting."""
    nx, ny = 9, 6
    rng = np.random.default_rng(2)
    ex = np.exp(rng.standard_normal(nx))
    eps = np.tile(ex, (ny, 1))
    Rf = 0.5 * (1.0 / ex[:-1] + 1.0 / ex[1:])
    prof = np.concatenate([[0.0], np.cumsum(Rf)]) / Rf.sum()
    g = np.tile(prof, (ny, 1))
    u = O.solve(nx, ny, eps, np.zeros((1, (nx - 2) * (ny - 2))), g)
    assert np.max(np.abs(u.reshape(ny - 2, nx - 2) - g[1:-1, 1:-1])) < 1e-14


def test_manufactured_second_order():
    """div(eps grad u) = f with smooth eps = 1 + sin(pi x) cos(pi y)/2 and
    u = sin(pi x) sin(pi y): the Eq. (6) error falls by ~4 per halving of h."""
    def case(n):
        h = 1.0 / (n - 1)
        X, Y = W.node_coords(n, n, h)
        pi = np.pi
        eps = 1.0 + 0.5 * np.sin(pi * X) * np.cos(pi * Y)
        ex = 0.5 * pi * np.cos(pi * X) * np.cos(pi * Y)
        ey = -0.5 * pi * np.sin(pi * X) * np.sin(pi * Y)
        ua = np.sin(pi * X) * np.sin(pi * Y)
        ux = pi * np.cos(pi * X) * np.sin(pi * Y)
        uy = pi * np.sin(pi * X) * np.cos(pi * Y)
        f = ex * ux + ey * uy - 2 * pi * pi * eps * ua
        rho = f[1:-1, 1:-1].reshape(1, -1)
        b = O.rhs_from_charge(n, n, h, eps, rho)
        u = O.solve(n, n, eps, b)
        return O.rel_error_eq6(u, ua[1:-1, 1:-1].reshape(1, -1))
    e = [case(n) for n in (17, 33, 65)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, e
    assert e[2] < 1e-3


# ---------------------------------------------------------------- invariants


def test_symmetric_conservative_form():
    nx, ny = 7, 6
    eps = W.eps_lognormal(nx, ny, seed=3)
    L, S, d = O.interior_operator(nx, ny, eps)
    assert np.array_equal(S, S.T)
    assert np.allclose(L, S / d[:, None], rtol=0, atol=0)
    A = O.assemble_full(nx, ny, eps)
    idx = [i * nx + j for i in range(1, ny - 1) for j in range(1, nx - 1)]
    assert np.max(np.abs(A[np.ix_(idx, idx)] - L)) < 1e-15
    # eps = 1 -> every weight is exactly 0.25 (Fig. 3)
    L1, _, d1 = O.interior_operator(nx, ny)
    off = L1[~np.eye(L1.shape[0], dtype=bool)]
    assert set(np.unique(off)) <= {0.0, -0.25}
    assert np.all(d1 == 4.0)


def test_inverse_nonnegative_m_matrix():
    nx, ny = 10, 8
    eps = W.eps_lognormal(nx, ny, seed=4)
    Linv = O.interior_inverse(nx, ny, eps)
    assert Linv.min() > 0.0


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 5), (5, 4), (6, 6), (3, 5)])
def test_brute_force_against_lapack(nx, ny):
    eps = W.eps_lognormal(nx, ny, seed=nx * 10 + ny)
    rng = np.random.default_rng(nx + ny)
    b = rng.standard_normal((3, (nx - 2) * (ny - 2)))
    L, _, _ = O.interior_operator(nx, ny, eps)
    ref = np.linalg.solve(L, b.T).T
    u = O.solve(nx, ny, eps, b, route="dense")
    assert np.max(np.abs(u - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(O.lu_inverse(L) - np.linalg.inv(L))) < 1e-13 * np.max(np.abs(np.linalg.inv(L)))
    r = O.residual(nx, ny, eps, b, u)
    assert np.max(np.abs(r)) < 1e-14 * np.max(np.abs(b))


def test_lu_partial_pivoting_permutes():
    """The dense LU needs its row exchanges on a matrix with a zero leading
    pivot, and still reproduces LAPACK."""
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    assert np.max(np.abs(O.lu_inverse(A) - np.linalg.inv(A))) < 1e-15


def test_band_route_matches_dense():
    nx, ny = 24, 19
    eps = W.eps_fourier(nx, ny, 1.0 / 23, seed=1)
    rng = np.random.default_rng(9)
    b = rng.standard_normal((4, (nx - 2) * (ny - 2)))
    ud = O.solve(nx, ny, eps, b, route="dense")
    ub = O.solve(nx, ny, eps, b, route="band")
    assert O.rel_error_eq6(ub, ud) < 1e-13
    Li_d = O.interior_inverse(nx, ny, eps, "dense")
    Li_b = O.interior_inverse(nx, ny, eps, "band")
    assert np.max(np.abs(Li_b - Li_d)) < 1e-13 * np.max(np.abs(Li_d))


def test_band_route_matches_lapack_50():
    """The 50x50 grid (48^2 unknowns): band LU against LAPACK's dense solve."""
    n = 50
    h = 1.0 / (n - 1)
    eps = W.eps_fourier(n, n, h, seed=1)
    rho = W.gaussian_blobs(n, n, h, seed=0)
    b = O.rhs_from_charge(n, n, h, eps, rho)
    L, _, _ = O.interior_operator(n, n, eps)
    ref = np.linalg.solve(L, b.T).T
    ub = O.solve(n, n, eps, b, route="band")
    assert O.rel_error_eq6(ub, ref) < 1e-13


# ---------------------------------------------------------------- adjoint


def test_adjoint_against_central_differences():
    """dLoss/db and dLoss/deps of Loss = 0.5 ||u - u_t||^2, u = L(eps)^-1 b,
    against FP64 central differences of the oracle's own solve."""
    nx, ny = 7, 6
    eps = W.eps_lognormal(nx, ny, seed=7)
    rng = np.random.default_rng(8)
    n = (nx - 2) * (ny - 2)
    b = rng.standard_normal((2, n))
    ut = rng.standard_normal((2, n))

    def loss(e, bb):
        u = O.solve(nx, ny, e, bb, route="dense")
        return 0.5 * np.sum((u - ut) ** 2)

    u0 = O.solve(nx, ny, eps, b, route="dense")
    u, db, deps = O.adjoint_gradients(nx, ny, eps, b, u0 - ut)
    assert np.max(np.abs(u - u0)) < 1e-15 * np.max(np.abs(u0)) + 1e-300
    for i in range(ny):
        for j in range(nx):
            if (i in (0, ny - 1)) and (j in (0, nx - 1)):
                assert deps[i, j] == 0.0     # corner nodes touch no interior face
                continue
            st = 1e-6 * eps[i, j]
            ep, em = eps.copy(), eps.copy()
            ep[i, j] += st
            em[i, j] -= st
            fd = (loss(ep, b) - loss(em, b)) / (2 * st)
            assert abs(fd - deps[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, deps[i, j])
    for c in range(2):
        for p in range(0, n, 3):
            bp, bm = b.copy(), b.copy()
            bp[c, p] += 1e-6
            bm[c, p] -= 1e-6
            fd = (loss(eps, bp) - loss(eps, bm)) / 2e-6
            assert abs(fd - db[c, p]) <= 1e-6 * max(1.0, abs(fd))


def test_rhs_from_charge_eps1():
    """At eps = 1 the right-hand side is -h^2 rho / 4 (the factor Table 1
    needs; the printed Eq. 2 drops the 1/4)."""
    n, h = 6, 0.2
    rho = np.arange(16.0)
    assert np.allclose(O.rhs_from_charge(n, n, h, None, rho), -h * h * rho / 4, rtol=1e-15, atol=0)
