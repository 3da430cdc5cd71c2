"""Pins of the 3-D oracle (oracle/pide_oracle3d.py) against facts fixed by the
mathematics: the discrete sine transform closed form, symmetry and
nonnegativity, exact harmonic data, second-order convergence, a brute-force
solve of the full system with identity boundary rows, band = dense."""
import numpy as np
import pytest

from oracle import pide_oracle3d as O3


def _lognormal(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return np.exp(0.5 * rng.standard_normal((nz, ny, nx)))


def _dst_inverse(nx, ny, nz):
    """L^-1 at eps = 1 from the 3-D sine basis: eigenvalues
    1 - (cos(a pi/(mx+1)) + cos(b pi/(my+1)) + cos(c pi/(mz+1))) / 3."""
    def basis(m):
        i = np.arange(1, m + 1)
        return np.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(i, i) / (m + 1)), \
            np.cos(np.pi * i / (m + 1))
    (Vx, cx), (Vy, cy), (Vz, cz) = basis(nx - 2), basis(ny - 2), basis(nz - 2)
    lam = 1.0 - (cz[:, None, None] + cy[None, :, None] + cx[None, None, :]) / 3.0
    V = np.kron(Vz, np.kron(Vy, Vx))          # x fastest
    return V @ np.diag(1.0 / lam.reshape(-1)) @ V.T


@pytest.mark.parametrize("dims", [(6, 5, 7), (3, 4, 5), (5, 3, 3)])
def test_dst_closed_form(dims):
    nx, ny, nz = dims
    A = O3.interior_inverse(nx, ny, nz)
    ref = _dst_inverse(nx, ny, nz)
    assert np.max(np.abs(A - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_weights_at_eps_one_are_one_sixth():
    L, S, d = O3.interior_operator(5, 5, 5)
    assert np.allclose(d, 6.0)
    p = O3.interior_index(2, 2, 2, 5, 5)          # the centre node: all six neighbours interior
    off = np.sort(L[p][L[p] != 0])
    assert np.allclose(off, [-1 / 6] * 6 + [1.0])


def test_symmetry_and_nonnegative_inverse():
    nx, ny, nz = 7, 6, 5
    eps = _lognormal(nx, ny, nz, 1)
    L, S, d = O3.interior_operator(nx, ny, nz, eps)
    assert np.max(np.abs(S - S.T)) == 0.0
    assert np.allclose(d[:, None] * L, S, rtol=0, atol=1e-15 * np.max(np.abs(S)))
    Linv = O3.interior_inverse(nx, ny, nz, eps)
    assert np.min(Linv) >= -1e-15
    # S^-1 = L^-1 D^-1 is symmetric
    Sinv = Linv / d[None, :]
    assert np.max(np.abs(Sinv - Sinv.T)) <= 1e-13 * np.max(np.abs(Sinv))


@pytest.mark.parametrize("func", ["linear", "quadratic"])
def test_harmonic_boundary_data_is_exact(func):
    """At eps = 1 the 7-point stencil is exact on harmonic polynomials of
    degree <= 2: with b = 0 and those boundary values the discrete solution
    equals the function at every interior node."""
    nx, ny, nz = 7, 6, 8
    h = 1.0 / 6
    z, y, x = np.meshgrid(h * np.arange(nz), h * np.arange(ny), h * np.arange(nx), indexing="ij")
    g = 1 + x + 2 * y - 3 * z if func == "linear" else x * x + y * y - 2 * z * z + x * y - y * z
    n = (nx - 2) * (ny - 2) * (nz - 2)
    u = O3.solve(nx, ny, nz, None, np.zeros((1, n)), g)
    assert np.max(np.abs(u[0] - g[1:-1, 1:-1, 1:-1].reshape(-1))) <= 1e-13 * np.max(np.abs(g))


def test_full_system_brute_force():
    """The full (nx ny nz)^2 system with identity rows at boundary nodes,
    assembled independently here and solved by LAPACK, has the oracle's
    interior solution for random b and boundary values."""
    nx, ny, nz = 4, 5, 6
    eps = _lognormal(nx, ny, nz, 2)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((nz, ny, nx))
    n = (nx - 2) * (ny - 2) * (nz - 2)
    b = rng.standard_normal(n)
    N = nx * ny * nz
    A = np.eye(N)
    rhs = g.reshape(-1).copy()
    for l in range(1, nz - 1):
        for i in range(1, ny - 1):
            for j in range(1, nx - 1):
                P = (l * ny + i) * nx + j
                faces = []
                for dz, dy, dx in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
                    e0, e1 = eps[l, i, j], eps[l + dz, i + dy, j + dx]
                    faces.append((((l + dz) * ny + (i + dy)) * nx + (j + dx), 2 * e0 * e1 / (e0 + e1)))
                tot = sum(f for _, f in faces)
                for Q, f in faces:
                    A[P, Q] -= f / tot
                rhs[P] = b[O3.interior_index(l, i, j, nx, ny)]
    full = np.linalg.solve(A, rhs).reshape(nz, ny, nx)
    u = O3.solve(nx, ny, nz, eps, b[None, :], g)[0]
    assert np.max(np.abs(u - full[1:-1, 1:-1, 1:-1].reshape(-1))) <= 1e-12 * np.max(np.abs(full))


def test_band_equals_dense_and_residual():
    nx, ny, nz = 7, 6, 8
    eps = _lognormal(nx, ny, nz, 4)
    rng = np.random.default_rng(5)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    b = rng.standard_normal((3, n))
    ud = O3.solve(nx, ny, nz, eps, b, route="dense")
    ub = O3.solve(nx, ny, nz, eps, b, route="band")
    assert np.max(np.abs(ud - ub)) <= 1e-12 * np.max(np.abs(ud))
    L, _, _ = O3.interior_operator(nx, ny, nz, eps)
    assert np.max(np.abs(b - (L @ ub.T).T)) <= 1e-13 * np.max(np.abs(b))
    r = O3.residual(nx, ny, nz, eps, b, ub)
    assert np.max(np.abs(r)) <= 1e-13 * np.max(np.abs(b))
    u = rng.standard_normal((2, n))
    assert np.allclose(O3.residual(nx, ny, nz, eps, b[:2], u), b[:2] - (L @ u.T).T, rtol=0,
                       atol=1e-14 * np.max(np.abs(u)))


def test_second_order_convergence():
    """div(eps grad u) = rho with u = sin(pi x) sin(pi y) sin(pi z) and
    eps = 1 + x y z / 2: the error falls ~4x when h halves."""
    def err(N):
        h = 1.0 / (N - 1)
        z, y, x = np.meshgrid(h * np.arange(N), h * np.arange(N), h * np.arange(N), indexing="ij")
        eps = 1 + 0.5 * x * y * z
        s, c = np.sin, np.cos
        u = s(np.pi * x) * s(np.pi * y) * s(np.pi * z)
        grad_eps_dot_grad_u = 0.5 * np.pi * (y * z * c(np.pi * x) * s(np.pi * y) * s(np.pi * z)
                                             + x * z * s(np.pi * x) * c(np.pi * y) * s(np.pi * z)
                                             + x * y * s(np.pi * x) * s(np.pi * y) * c(np.pi * z))
        rho = -3 * np.pi ** 2 * eps * u + grad_eps_dot_grad_u
        b = O3.rhs_from_charge(N, N, N, h, eps, rho[1:-1, 1:-1, 1:-1].reshape(1, -1))
        un = O3.solve(N, N, N, eps, b, route="band")[0]
        return np.max(np.abs(un - u[1:-1, 1:-1, 1:-1].reshape(-1))) / np.max(np.abs(u))
    e1, e2 = err(9), err(17)
    assert 3.5 <= e1 / e2 <= 4.6, (e1, e2)


def test_adjoint_against_central_differences():
    """dLoss/db and dLoss/deps of Loss = 0.5 ||u - u_t||^2, u = L(eps)^-1 b,
    against FP64 central differences of the oracle's own solve."""
    nx, ny, nz = 5, 4, 5
    eps = _lognormal(nx, ny, nz, 11)
    rng = np.random.default_rng(12)
    n = (nx - 2) * (ny - 2) * (nz - 2)
    b = rng.standard_normal((2, n))
    ut = rng.standard_normal((2, n))

    def loss(e, bb):
        u = O3.solve(nx, ny, nz, e, bb, route="dense")
        return 0.5 * np.sum((u - ut) ** 2)

    u0 = O3.solve(nx, ny, nz, eps, b, route="dense")
    u, db, deps = O3.adjoint_gradients(nx, ny, nz, eps, b, u0 - ut)
    assert np.max(np.abs(u - u0)) < 1e-13 * np.max(np.abs(u0))
    for l in range(nz):
        for i in range(ny):
            for j in range(nx):
                st = 1e-6 * eps[l, i, j]
                ep, em = eps.copy(), eps.copy()
                ep[l, i, j] += st
                em[l, i, j] -= st
                fd = (loss(ep, b) - loss(em, b)) / (2 * st)
                assert abs(fd - deps[l, i, j]) <= 1e-6 * max(1.0, abs(fd)), (l, i, j, fd, deps[l, i, j])
    for c in range(2):
        for p in range(0, n, 2):
            bp, bm = b.copy(), b.copy()
            bp[c, p] += 1e-6
            bm[c, p] -= 1e-6
            fd = (loss(eps, bp) - loss(eps, bm)) / 2e-6
            assert abs(fd - db[c, p]) <= 1e-6 * max(1.0, abs(fd))
