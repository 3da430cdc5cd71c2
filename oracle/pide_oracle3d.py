"""Plain, slow FP64 CPU oracle for the three-dimensional operator.

TEST INFRASTRUCTURE ONLY, like ``pide_oracle``: only the tests, the smoke
entry and the benchmark's CPU leg may import it; it shares no code with the
CUDA library.

The paper states its problem for N grid points in general and works the
two-dimensional case (Eq. 2, Fig. 3); this module is the same construction on
an nx x ny x nz node grid: the 7-point flux-form operator of Eq. (1)
(permittivity on the faces by harmonic mean of the two node values, each
interior row divided by its total face permittivity as in Eq. 3, so that at
eps = 1 every weight is 1/6), identity rows at boundary nodes carrying the
boundary value, nodes ordered with x fastest, then y, then z.  The solution
steps are the paper's: assemble, invert by a standard method (dense LU with
partial pivoting, or the same LU restricted to the band of half-width
(nx-2)(ny-2) with no pivoting on the diagonally dominant operator), multiply.

Pins (tests/test_oracle3d.py): the 3-D discrete sine transform closed form at
eps = 1, symmetry of D*L, nonnegativity of L^-1, exact reproduction of
harmonic linear and quadratic boundary data at eps = 1 (the 7-point stencil
is exact on them), second-order convergence on a manufactured solution with
smooth eps, the residual of the solve, banded-vs-dense agreement.
"""
from __future__ import annotations

import numpy as np

from oracle.pide_oracle import band_lu, band_solve, harmonic, lu_inverse

# ---------------------------------------------------------------------------
# Grid bookkeeping
# ---------------------------------------------------------------------------

# neighbour offsets (dz, dy, dx) in the face order W, E, S, N, D, U
OFFSETS = ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0))


def is_boundary(l: int, i: int, j: int, nx: int, ny: int, nz: int) -> bool:
    return l == 0 or l == nz - 1 or i == 0 or i == ny - 1 or j == 0 or j == nx - 1


def interior_index(l: int, i: int, j: int, nx: int, ny: int) -> int:
    """Interior node (l, i, j) -> p, x fastest."""
    mx, my = nx - 2, ny - 2
    return ((l - 1) * my + (i - 1)) * mx + (j - 1)


def node_face_weights(eps: np.ndarray, l: int, i: int, j: int):
    """((neighbour), eps_face) for the six faces of interior node (l, i, j)."""
    out = []
    for dz, dy, dx in OFFSETS:
        a, b, c = l + dz, i + dy, j + dx
        out.append(((a, b, c), harmonic(eps[l, i, j], eps[a, b, c])))
    return out


def _eps(nx, ny, nz, eps):
    return np.ones((nz, ny, nx)) if eps is None else np.asarray(eps, dtype=np.float64)


# ---------------------------------------------------------------------------
# Step 1: assembly
# ---------------------------------------------------------------------------


def interior_operator(nx: int, ny: int, nz: int, eps: np.ndarray | None = None):
    """(L, S, d): L = I - W on the interior (boundary columns removed),
    S the symmetric conservative form (S_pp = sum of the node's face eps,
    S_pq = -eps_pq), d the diagonal of S, L = diag(d)^-1 S."""
    eps = _eps(nx, ny, nz, eps)
    mx, my, mz = nx - 2, ny - 2, nz - 2
    n = mx * my * mz
    S = np.zeros((n, n))
    for l in range(1, nz - 1):
        for i in range(1, ny - 1):
            for j in range(1, nx - 1):
                p = interior_index(l, i, j, nx, ny)
                for (a, b, c), e in node_face_weights(eps, l, i, j):
                    S[p, p] += e
                    if not is_boundary(a, b, c, nx, ny, nz):
                        S[p, interior_index(a, b, c, nx, ny)] = -e
    d = np.diag(S).copy()
    return S / d[:, None], S, d


def diagonal_d(nx: int, ny: int, nz: int, eps: np.ndarray | None) -> np.ndarray:
    eps = _eps(nx, ny, nz, eps)
    mx, my, mz = nx - 2, ny - 2, nz - 2
    d = np.zeros(mx * my * mz)
    for l in range(1, nz - 1):
        for i in range(1, ny - 1):
            for j in range(1, nx - 1):
                d[interior_index(l, i, j, nx, ny)] = sum(
                    e for _, e in node_face_weights(eps, l, i, j))
    return d


def boundary_lift(nx: int, ny: int, nz: int, eps: np.ndarray | None, g: np.ndarray) -> np.ndarray:
    """sum over boundary neighbours q of w_pq g_q (the identity rows' values
    moved to the right side of the interior rows)."""
    eps = _eps(nx, ny, nz, eps)
    mx, my, mz = nx - 2, ny - 2, nz - 2
    out = np.zeros(mx * my * mz)
    for l in range(1, nz - 1):
        for i in range(1, ny - 1):
            for j in range(1, nx - 1):
                p = interior_index(l, i, j, nx, ny)
                fw = node_face_weights(eps, l, i, j)
                tot = sum(e for _, e in fw)
                for (a, b, c), e in fw:
                    if is_boundary(a, b, c, nx, ny, nz):
                        out[p] += e / tot * g[a, b, c]
    return out


def rhs_from_charge(nx: int, ny: int, nz: int, h: float, eps: np.ndarray | None,
                    rho: np.ndarray) -> np.ndarray:
    """b = -h^2 rho / d: the interior right side of div(eps grad u) = rho (the
    sign of Eq. 4's Laplace form) after dividing each row by its total face
    permittivity."""
    return -h * h * np.atleast_2d(rho) / diagonal_d(nx, ny, nz, eps)[None, :]


def band_of(nx: int, ny: int, nz: int, eps: np.ndarray | None):
    """L in band storage, half-width w = (nx-2)(ny-2) (the distance between
    neighbours in z): band[p, w + c] = L[p, p + c]."""
    eps = _eps(nx, ny, nz, eps)
    mx, my, mz = nx - 2, ny - 2, nz - 2
    n, w = mx * my * mz, mx * my
    band = np.zeros((n, 2 * w + 1))
    for l in range(1, nz - 1):
        for i in range(1, ny - 1):
            for j in range(1, nx - 1):
                p = interior_index(l, i, j, nx, ny)
                fw = node_face_weights(eps, l, i, j)
                tot = sum(e for _, e in fw)
                band[p, w] = 1.0
                for (a, b, c), e in fw:
                    if not is_boundary(a, b, c, nx, ny, nz):
                        band[p, w + (interior_index(a, b, c, nx, ny) - p)] = -e / tot
    return band


# ---------------------------------------------------------------------------
# Steps 2 and 3
# ---------------------------------------------------------------------------


def interior_inverse(nx: int, ny: int, nz: int, eps: np.ndarray | None = None,
                     route: str = "dense") -> np.ndarray:
    """L^-1 by dense LU (partial pivoting) or by band LU."""
    if route == "dense":
        L, _, _ = interior_operator(nx, ny, nz, eps)
        return lu_inverse(L)
    F = band_lu(band_of(nx, ny, nz, eps))
    return band_solve(F, np.eye(F.shape[0]))


class BandSolver:
    """Factor L once (band LU), then solve any number of right-hand sides."""

    def __init__(self, nx: int, ny: int, nz: int, eps: np.ndarray | None = None):
        self.F = band_lu(band_of(nx, ny, nz, eps))

    def solve(self, b: np.ndarray) -> np.ndarray:
        return band_solve(self.F, np.atleast_2d(b).T).T


def solve(nx: int, ny: int, nz: int, eps: np.ndarray | None, b: np.ndarray,
          g: np.ndarray | None = None, route: str = "auto") -> np.ndarray:
    """Interior u of the 3-D system for right-hand sides b ([B][n]) and
    boundary values g ([nz][ny][nx], default zero)."""
    b2 = np.atleast_2d(np.asarray(b, dtype=np.float64))
    if g is not None:
        b2 = b2 + boundary_lift(nx, ny, nz, eps, g)[None, :]
    n = (nx - 2) * (ny - 2) * (nz - 2)
    if route == "auto":
        route = "dense" if n <= 700 else "band"
    if route == "dense":
        return (interior_inverse(nx, ny, nz, eps, "dense") @ b2.T).T
    return BandSolver(nx, ny, nz, eps).solve(b2)


def residual(nx: int, ny: int, nz: int, eps: np.ndarray | None, b: np.ndarray,
             u: np.ndarray) -> np.ndarray:
    """r = b - L u (zero boundary values), from the band form."""
    band = band_of(nx, ny, nz, eps)
    n, wid = band.shape
    w = (wid - 1) // 2
    U = np.atleast_2d(u)
    Lu = np.zeros_like(U)
    for c in sorted({-w, -(nx - 2), -1, 0, 1, nx - 2, w}):
        lo, hi = max(0, -c), min(n, n - c)
        Lu[:, lo:hi] += band[lo:hi, w + c] * U[:, lo + c:hi + c]
    return np.atleast_2d(b) - Lu


# ---------------------------------------------------------------------------
# Adjoint (not in the paper; the same derivation as the 2-D oracle's)
# ---------------------------------------------------------------------------


def adjoint_gradients(nx: int, ny: int, nz: int, eps: np.ndarray, b: np.ndarray,
                      gout: np.ndarray):
    """Gradients of Loss(u), u = L(eps)^-1 b with b held fixed and zero
    boundary values: mu = S^-1 gout (S = D L symmetric), dLoss/db = D mu, and
    for a face of permittivity e_f between nodes p and q
        dLoss/de_f = mu_p b_p + mu_q b_q - (mu_p - mu_q)(u_p - u_q)
    (a boundary node contributes mu = 0, no b term, u = 0), chained to the
    node values through d e_f / d eps_a = 2 eps_b^2 / (eps_a + eps_b)^2.
    Returns (u, dLoss/db, dLoss/deps[nz][ny][nx])."""
    eps = _eps(nx, ny, nz, eps)
    _, S, d = interior_operator(nx, ny, nz, eps)
    b2 = np.atleast_2d(b)
    G = np.atleast_2d(gout)
    u = (np.linalg.solve(S, (b2 * d[None, :]).T)).T          # L u = b  <=>  S u = D b
    mu = np.linalg.solve(S, G.T).T
    db = mu * d[None, :]
    deps = np.zeros((nz, ny, nx))

    def val(arr, l, i, j, c):
        return arr[c, interior_index(l, i, j, nx, ny)]

    for l in range(nz):
        for i in range(ny):
            for j in range(nx):
                for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):   # each face once
                    l2, i2, j2 = l + dz, i + dy, j + dx
                    if l2 >= nz or i2 >= ny or j2 >= nx:
                        continue
                    ba = is_boundary(l, i, j, nx, ny, nz)
                    bb = is_boundary(l2, i2, j2, nx, ny, nz)
                    if ba and bb:
                        continue
                    tot = 0.0
                    for c in range(b2.shape[0]):
                        mu_a = 0.0 if ba else val(mu, l, i, j, c)
                        mu_b = 0.0 if bb else val(mu, l2, i2, j2, c)
                        u_a = 0.0 if ba else val(u, l, i, j, c)
                        u_b = 0.0 if bb else val(u, l2, i2, j2, c)
                        b_a = 0.0 if ba else val(b2, l, i, j, c)
                        b_b = 0.0 if bb else val(b2, l2, i2, j2, c)
                        tot += mu_a * b_a + mu_b * b_b - (mu_a - mu_b) * (u_a - u_b)
                    ea, eb = eps[l, i, j], eps[l2, i2, j2]
                    deps[l, i, j] += tot * 2 * eb * eb / (ea + eb) ** 2
                    deps[l2, i2, j2] += tot * 2 * ea * ea / (ea + eb) ** 2
    return u, db, deps
