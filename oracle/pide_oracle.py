"""Plain, slow FP64 CPU oracle for the dense-inverse Poisson apply.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke entry and
the CPU-baseline leg of the benchmark may import this module.  It shares no
code with the CUDA library: nothing here is imported by the product package,
and this module imports nothing from it.

What it computes (Dourbal & Pekker, "A New Numerical Method for Fast Solution
of Partial Integro-Differential Equations"):

* Eq. (2) / Fig. 3: the 5-point system on an nx x ny node grid with spacing h,
  boundary nodes as identity rows whose right-hand side is the boundary
  value, nodes ordered row by row with j (x index) fastest.
* Eq. (3): the general form u_p - sum_q w_pq u_q = b_p.  For variable
  permittivity the weights come from the conservative flux form of Eq. (1):
  face permittivity by harmonic mean of the two node values, w_pq =
  eps_pq / sum_q' eps_pq'.  At eps = 1 every weight is 0.25 (Fig. 3).
* "The solution steps": (1) assemble the matrix, (2) invert it by a standard
  method -- here dense LU with partial pivoting, or for large grids the same
  LU restricted to the band (no pivoting; the operator is diagonally
  dominant), (3) multiply the inverse by the right-hand side.
* Eq. (6): relative max-norm error.
* Table 1's experiment: round the entries of the inverse to k decimals.
* The adjoint of u = L(eps)^-1 b (not in the paper; the gradient formula is
  derived here from differentiating L u = b, see ``adjoint_gradients``).
* The stored formats of the inverse written out (not in the paper, which
  rounds to decimals): bfloat16, float32, e4m3 and binary16 rounding, and the
  quantisers built on them (per-row e4m3 scales, power-of-two FP16 row and
  column scales, the e4m3 correction term of a BF16 or FP16 store), so that
  tests can form the exact product of the GPU's own roundings.

Precision: float64 throughout.  Loops are plain Python over one index with
numpy vector operations inside; there is no blocking or reordering beyond the
textbook algorithms named above.

Pins (tests/test_oracle.py): Fig. 3 bit-exact, Table 1 (24 of 25 cells,
which also pins Eq. (6): ``table1_row`` measures its error through
``rel_error_eq6``), a hand-computed multi-column Eq. (6) case whose worst
column is not the one with the largest |u|, the 2-D discrete sine transform
closed form at eps = 1, second-order convergence on a manufactured solution
with smooth eps, symmetry of D*L, nonnegativity of L^-1, brute force against
LAPACK on tiny grids, banded-vs-dense agreement, and central finite
differences for the adjoint; the roundings against torch's conversions and
exact ties, the quantisers by their error bounds and scale ranges, the
two-term e4m3 quantiser by its 2^-8 error bound, the range of its lo term and
lo = 0 on rows exact in e4m3 (tests/test_capi.py).  tests/test_oracle_pins.py
plants plausible mistakes in copies of Eq. (6) and of the two-term quantiser
and checks that these pins reject every one of them.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Grid bookkeeping (Eq. 2, Fig. 2/3)
# ---------------------------------------------------------------------------


def full_index(i: int, j: int, nx: int) -> int:
    """0-based node (i, j) -> row of the full Fig. 3 system (j fastest)."""
    return i * nx + j


def is_boundary(i: int, j: int, nx: int, ny: int) -> bool:
    return i == 0 or j == 0 or i == ny - 1 or j == nx - 1


def harmonic(a: float, b: float) -> float:
    """Face permittivity between two nodes (harmonic mean)."""
    return 2.0 * a * b / (a + b)


def neighbours(i: int, j: int):
    """The four 5-point neighbours of node (i, j) in the order of Eq. (2)."""
    return ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1))


def face_eps(eps: np.ndarray):
    """Face permittivities: ex[i][j] between (i,j),(i,j+1); ey[i][j] between
    (i,j),(i+1,j).  Harmonic mean of the node values."""
    ex = 2.0 * eps[:, :-1] * eps[:, 1:] / (eps[:, :-1] + eps[:, 1:])
    ey = 2.0 * eps[:-1, :] * eps[1:, :] / (eps[:-1, :] + eps[1:, :])
    return ex, ey


def node_face_weights(eps: np.ndarray, i: int, j: int):
    """(neighbour, eps_face) pairs of interior node (i, j)."""
    out = []
    for (a, b) in neighbours(i, j):
        out.append(((a, b), harmonic(eps[i, j], eps[a, b])))
    return out


# ---------------------------------------------------------------------------
# Step 1: assembly
# ---------------------------------------------------------------------------


def assemble_full(nx: int, ny: int, eps: np.ndarray | None = None) -> np.ndarray:
    """The full N x N matrix of Fig. 3 / Eq. (3), N = nx*ny.

    Boundary rows are identity rows.  Interior row p: 1 on the diagonal and
    -w_pq at each of the four neighbours, w_pq = eps_pq / sum eps_pq'.
    """
    if eps is None:
        eps = np.ones((ny, nx))
    N = nx * ny
    A = np.zeros((N, N))
    for i in range(ny):
        for j in range(nx):
            p = full_index(i, j, nx)
            A[p, p] = 1.0
            if is_boundary(i, j, nx, ny):
                continue
            fw = node_face_weights(eps, i, j)
            tot = sum(e for _, e in fw)
            for (a, b), e in fw:
                A[p, full_index(a, b, nx)] = -e / tot
    return A


def full_rhs(nx: int, ny: int, b_int: np.ndarray, g: np.ndarray | None = None) -> np.ndarray:
    """Right-hand side of Fig. 3: boundary value at boundary rows, b at
    interior rows.  ``b_int`` is [..., n_interior] (j fastest)."""
    if g is None:
        g = np.zeros((ny, nx))
    lead = b_int.shape[:-1]
    out = np.broadcast_to(g, lead + (ny, nx)).copy()
    out[..., 1:-1, 1:-1] = b_int.reshape(lead + (ny - 2, nx - 2))
    return out.reshape(lead + (nx * ny,))


def interior_operator(nx: int, ny: int, eps: np.ndarray | None = None):
    """Interior block of Eq. (3) in two equivalent forms.

    Returns (L, S, d) with L = I - W (the interior rows of Fig. 3 with the
    boundary columns removed), S the symmetric conservative form
    (S_pp = sum of the node's face eps, S_pq = -eps_pq) and d the diagonal of
    S, so that L = diag(d)^-1 S.
    """
    if eps is None:
        eps = np.ones((ny, nx))
    mx, my = nx - 2, ny - 2
    n = mx * my
    S = np.zeros((n, n))
    for i in range(1, ny - 1):
        for j in range(1, nx - 1):
            p = (i - 1) * mx + (j - 1)
            for (a, b), e in node_face_weights(eps, i, j):
                S[p, p] += e
                if not is_boundary(a, b, nx, ny):
                    S[p, (a - 1) * mx + (b - 1)] = -e
    d = np.diag(S).copy()
    L = S / d[:, None]
    return L, S, d


def boundary_lift(nx: int, ny: int, eps: np.ndarray | None, g: np.ndarray) -> np.ndarray:
    """Interior contribution of boundary values: sum over boundary
    neighbours q of w_pq g_q (moving Fig. 3's boundary columns to the right)."""
    if eps is None:
        eps = np.ones((ny, nx))
    mx, my = nx - 2, ny - 2
    out = np.zeros(mx * my)
    for i in range(1, ny - 1):
        for j in range(1, nx - 1):
            p = (i - 1) * mx + (j - 1)
            fw = node_face_weights(eps, i, j)
            tot = sum(e for _, e in fw)
            for (a, b), e in fw:
                if is_boundary(a, b, nx, ny):
                    out[p] += e / tot * g[a, b]
    return out


def rhs_from_charge(nx: int, ny: int, h: float, eps: np.ndarray | None,
                    rho: np.ndarray) -> np.ndarray:
    """Eq. (1) -> Eq. (3) right-hand side: b_p = -h^2 rho_p / sum_q eps_pq.

    Summing the face fluxes eps_pq (u_q - u_p)/h^2 = rho_p and dividing by the
    node's total face permittivity gives Eq. (3) with b = -h^2 rho / d; at
    eps = 1 this is -h^2 rho / 4 (the factor Table 1 needs).
    """
    if eps is None:
        eps = np.ones((ny, nx))
    return -h * h * rho / diagonal_d(nx, ny, eps)


def diagonal_d(nx: int, ny: int, eps: np.ndarray) -> np.ndarray:
    """Only the diagonal d of S (cheap; avoids the dense n x n build)."""
    mx, my = nx - 2, ny - 2
    d = np.zeros(mx * my)
    for i in range(1, ny - 1):
        for j in range(1, nx - 1):
            d[(i - 1) * mx + (j - 1)] = sum(e for _, e in node_face_weights(eps, i, j))
    return d


# ---------------------------------------------------------------------------
# Step 2: inversion by LU
# ---------------------------------------------------------------------------


def lu_factor(A: np.ndarray):
    """Doolittle LU with partial pivoting: P A = L U, packed in one array."""
    LU = np.array(A, dtype=np.float64, copy=True)
    n = LU.shape[0]
    perm = np.arange(n)
    for k in range(n):
        r = k + int(np.argmax(np.abs(LU[k:, k])))
        if LU[r, k] == 0.0:
            raise np.linalg.LinAlgError("singular matrix")
        if r != k:
            LU[[k, r]] = LU[[r, k]]
            perm[[k, r]] = perm[[r, k]]
        LU[k + 1:, k] /= LU[k, k]
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
    return LU, perm


def lu_solve(LU: np.ndarray, perm: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B given P A = L U.  B is [n] or [n][k]."""
    X = np.array(B, dtype=np.float64)[perm]
    n = LU.shape[0]
    for i in range(n):                      # L y = P b (unit lower)
        X[i] -= LU[i, :i] @ X[:i]
    for i in range(n - 1, -1, -1):          # U x = y
        X[i] = (X[i] - LU[i, i + 1:] @ X[i + 1:]) / LU[i, i]
    return X


def lu_inverse(A: np.ndarray) -> np.ndarray:
    """Step 2 with a standard method: A^-1 from LU and the identity columns."""
    LU, perm = lu_factor(A)
    return lu_solve(LU, perm, np.eye(A.shape[0]))


def band_of(nx: int, ny: int, eps: np.ndarray | None):
    """The interior operator L = I - W in band storage.

    band[p, w + c] = L[p, p + c] for -w <= c <= w, w = nx - 2 (the distance
    between vertical neighbours).  Entries outside the band are zero.
    """
    if eps is None:
        eps = np.ones((ny, nx))
    mx, my = nx - 2, ny - 2
    n, w = mx * my, mx
    band = np.zeros((n, 2 * w + 1))
    for i in range(1, ny - 1):
        for j in range(1, nx - 1):
            p = (i - 1) * mx + (j - 1)
            fw = node_face_weights(eps, i, j)
            tot = sum(e for _, e in fw)
            band[p, w] = 1.0
            for (a, b), e in fw:
                if not is_boundary(a, b, nx, ny):
                    q = (a - 1) * mx + (b - 1)
                    band[p, w + (q - p)] = -e / tot
    return band


def band_lu(band: np.ndarray) -> np.ndarray:
    """LU without pivoting of a band matrix, kept in band storage.

    The same elimination as ``lu_factor`` restricted to the band: for a
    diagonally dominant matrix no pivoting is needed and no fill appears
    outside the band.  Multipliers overwrite the sub-diagonal part.
    """
    F = np.array(band, dtype=np.float64, copy=True)
    n, wid = F.shape
    w = (wid - 1) // 2
    flat = F.reshape(-1)
    st = flat.strides[0]
    for k in range(n):
        r = min(w, n - 1 - k)
        if r == 0:
            break
        piv = F[k, w]
        base = k * wid + w
        # element (k+dl, k+t) lives at flat index base + dl*(wid-1) + t
        mult = np.lib.stride_tricks.as_strided(
            flat[base + (wid - 1):], shape=(r,), strides=((wid - 1) * st,), writeable=True)
        mult /= piv
        urow = F[k, w + 1:w + 1 + w]
        sub = np.lib.stride_tricks.as_strided(
            flat[base + (wid - 1) + 1:], shape=(r, w), strides=((wid - 1) * st, st),
            writeable=True)
        sub -= np.outer(mult, urow)
    return F


def band_solve(F: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Forward and back substitution with the band LU factors.  B: [n] or [n][k]."""
    n, wid = F.shape
    w = (wid - 1) // 2
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(n):
        lo = max(0, i - w)
        if i > lo:
            X[i] -= F[i, w - (i - lo):w] @ X[lo:i]
    for i in range(n - 1, -1, -1):
        hi = min(n, i + w + 1)
        if hi > i + 1:
            X[i] -= F[i, w + 1:w + (hi - i)] @ X[i + 1:hi]
        X[i] /= F[i, w]
    return X


# ---------------------------------------------------------------------------
# Step 3: apply, and the error metric
# ---------------------------------------------------------------------------


def apply_inverse(Ainv: np.ndarray, b: np.ndarray) -> np.ndarray:
    """u = A^-1 b for every column.  b is [B][n] (one right-hand side per row)."""
    return (Ainv @ np.atleast_2d(b).T).T


def interior_inverse(nx: int, ny: int, eps: np.ndarray | None = None,
                     route: str = "dense") -> np.ndarray:
    """L^-1 for the interior block, by dense LU or band LU."""
    if route == "dense":
        L, _, _ = interior_operator(nx, ny, eps)
        return lu_inverse(L)
    F = band_lu(band_of(nx, ny, eps))
    n = F.shape[0]
    return band_solve(F, np.eye(n))


class BandSolver:
    """Factor L once (band LU), then solve for any number of columns."""

    def __init__(self, nx: int, ny: int, eps: np.ndarray | None = None):
        self.nx, self.ny = nx, ny
        self.F = band_lu(band_of(nx, ny, eps))

    def solve(self, b: np.ndarray) -> np.ndarray:
        b2 = np.atleast_2d(b)
        return band_solve(self.F, b2.T).T


def solve(nx: int, ny: int, eps: np.ndarray | None, b: np.ndarray,
          g: np.ndarray | None = None, route: str = "auto") -> np.ndarray:
    """The method's result: interior u of the Fig. 3 system for right-hand
    side b (interior, [B][n]) and boundary values g (default zero)."""
    b2 = np.atleast_2d(np.asarray(b, dtype=np.float64))
    if g is not None:
        b2 = b2 + boundary_lift(nx, ny, eps, g)[None, :]
    n = (nx - 2) * (ny - 2)
    if route == "auto":
        route = "dense" if n <= 900 else "band"
    if route == "dense":
        return apply_inverse(interior_inverse(nx, ny, eps, "dense"), b2)
    return BandSolver(nx, ny, eps).solve(b2)


def rel_error_eq6(u_num: np.ndarray, u_ref: np.ndarray) -> float:
    """Eq. (6): max |u_ref - u_num| / max |u_ref|, worst over columns."""
    a = np.atleast_2d(u_num)
    r = np.atleast_2d(u_ref)
    num = np.max(np.abs(a - r), axis=1)
    den = np.max(np.abs(r), axis=1)
    return float(np.max(num / den))


def residual(nx: int, ny: int, eps: np.ndarray | None, b: np.ndarray,
             u: np.ndarray) -> np.ndarray:
    """r = b - L u with L the interior block of Eq. (3) (zero boundary)."""
    band = band_of(nx, ny, eps)
    n, wid = band.shape
    w = (wid - 1) // 2
    U = np.atleast_2d(u)
    Lu = np.zeros_like(U)
    for c in range(-w, w + 1):
        lo, hi = max(0, -c), min(n, n - c)
        Lu[:, lo:hi] += band[lo:hi, w + c] * U[:, lo + c:hi + c]
    return np.atleast_2d(b) - Lu


# ---------------------------------------------------------------------------
# Table 1's experiment (Eqs. 4-6)
# ---------------------------------------------------------------------------


def eq4_source(x, y):
    """Right side of Eq. (4)."""
    return (12 * x ** 2 - 6 * x) * (y ** 3 - y ** 2) + (x ** 4 - x ** 3) * (6 * y - 2)


def eq5_exact(x, y):
    """Exact solution, Eq. (5)."""
    return (x ** 4 - x ** 3) * (y ** 3 - y ** 2)


def round_decimals(A: np.ndarray, k: int) -> np.ndarray:
    """Round every entry to k digits after the decimal point (nearest; ties
    away from zero)."""
    s = 10.0 ** k
    return np.sign(A) * np.floor(np.abs(A) * s + 0.5) / s


def table1_row(n: int, digits_list, route: str = "auto"):
    """One column of Table 1 (grid n x n on [0,1]^2): the Eq. (6) error over
    all nodes for each entry of ``digits_list`` (None = no rounding).

    Steps as in the paper's numerical example: build L for Eq. (4) with zero
    boundary values, invert it, round the inverse's entries, multiply by the
    right-hand side, compare with Eq. (5).
    """
    h = 1.0 / (n - 1)
    x = h * np.arange(n)
    X, Y = np.meshgrid(x, x)
    f = eq4_source(X, Y)[1:-1, 1:-1].reshape(-1)
    b = rhs_from_charge(n, n, h, None, f)
    if route == "auto":
        route = "dense" if (n - 2) ** 2 <= 900 else "band"
    Linv = interior_inverse(n, n, None, route)
    ua = eq5_exact(X, Y)
    out = []
    for digits in digits_list:
        M = Linv if digits is None else round_decimals(Linv, digits)
        u = np.zeros((n, n))
        u[1:-1, 1:-1] = (M @ b).reshape(n - 2, n - 2)
        # Eq. (6) over every node of the grid (boundary nodes carry u = 0 on both sides)
        out.append(rel_error_eq6(u.reshape(-1), ua.reshape(-1)))
    return out


# ---------------------------------------------------------------------------
# Adjoint (not in the paper)
# ---------------------------------------------------------------------------


def adjoint_gradients(nx: int, ny: int, eps: np.ndarray, b: np.ndarray,
                      gout: np.ndarray, g: np.ndarray | None = None):
    """Gradients of Loss(u) with u = L(eps)^-1 b, b held fixed.

    With L = D^-1 S (S symmetric), mu = S^-1 gout solves the adjoint system.
    Then dLoss/db = D mu, and differentiating L u = b in one face
    permittivity e_f between nodes p and q gives
        dLoss/de_f = mu_p b_p + mu_q b_q - (mu_p - mu_q)(u_p - u_q),
    where a boundary node contributes mu = 0, no b term and u = g.  The face
    value is the harmonic mean of its two nodes, d e_f / d eps_a =
    2 eps_b^2 / (eps_a + eps_b)^2.  Returns (u, dLoss/db, dLoss/deps[ny][nx]).
    """
    mx, my = nx - 2, ny - 2
    if g is None:
        g = np.zeros((ny, nx))
    L, S, d = interior_operator(nx, ny, eps)
    b2 = np.atleast_2d(b)
    G = np.atleast_2d(gout)
    u = solve(nx, ny, eps, b2, g, route="dense" if mx * my <= 900 else "band")
    Sinv_g = np.linalg.solve(S, G.T).T if mx * my <= 2500 else \
        BandSolver(nx, ny, eps).solve(G / d[None, :])
    mu = Sinv_g
    db = mu * d[None, :]
    deps = np.zeros((ny, nx))

    def val(arr, i, j, c):
        return arr[c, (i - 1) * mx + (j - 1)]

    faces = []
    for i in range(ny):
        for j in range(nx - 1):
            faces.append(((i, j), (i, j + 1)))
    for i in range(ny - 1):
        for j in range(nx):
            faces.append(((i, j), (i + 1, j)))
    for (pa, pb) in faces:
        ia, ja = pa
        ib, jb = pb
        ba, bb = is_boundary(ia, ja, nx, ny), is_boundary(ib, jb, nx, ny)
        if ba and bb:
            continue
        tot = 0.0
        for c in range(b2.shape[0]):
            mu_a = 0.0 if ba else val(mu, ia, ja, c)
            mu_b = 0.0 if bb else val(mu, ib, jb, c)
            u_a = g[ia, ja] if ba else val(u, ia, ja, c)
            u_b = g[ib, jb] if bb else val(u, ib, jb, c)
            b_a = 0.0 if ba else val(b2, ia, ja, c)
            b_b = 0.0 if bb else val(b2, ib, jb, c)
            tot += mu_a * b_a + mu_b * b_b - (mu_a - mu_b) * (u_a - u_b)
        ea, eb = eps[ia, ja], eps[ib, jb]
        deps[ia, ja] += tot * 2 * eb * eb / (ea + eb) ** 2
        deps[ib, jb] += tot * 2 * ea * ea / (ea + eb) ** 2
    return u, db, deps


# ---------------------------------------------------------------------------
# Binary rounding of the stored inverse (the GPU's analogue of Table 1's
# decimal rounding): round to nearest, ties to even, from float64.
# ---------------------------------------------------------------------------


def round_to_bits(x: np.ndarray, bits: int) -> np.ndarray:
    """Round each value to ``bits`` significant bits (nearest, ties to even),
    no exponent limit: x = m 2^e with 0.5 <= |m| < 1, m rounded to bits bits."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 2.0 ** bits) / 2.0 ** bits, e)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """bfloat16 value of each entry (8 significant bits; normal range only)."""
    return round_to_bits(x, 8)


def round_fp32(x: np.ndarray) -> np.ndarray:
    """float32 value of each entry (24 significant bits; normal range only)."""
    return round_to_bits(x, 24)


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """e4m3 (OCP FP8, 4 exponent bits, 3 mantissa bits, bias 7) value of each
    entry, nearest with ties to even, saturating at the largest finite 448:
    4 significant bits for |x| >= 2^-6, fixed quantum 2^-9 below (subnormals)."""
    x = np.asarray(x, dtype=np.float64)
    normal = round_to_bits(x, 4)
    sub = np.rint(x / 2.0 ** -9) * 2.0 ** -9
    out = np.where(np.abs(x) >= 2.0 ** -6, normal, sub)
    return np.clip(out, -448.0, 448.0)


def quantize_rows_e4m3(M: np.ndarray, two_terms: bool):
    """Per-row e4m3 storage of a matrix, the GPU's FP8 format written out:
    scale s_p = float32(max_q |M_pq| / 448); x = M / s in FP64, taken to
    float32, hi = e4m3(x); lo = e4m3(float32(x - hi)).  Returns (s, hi, lo)
    with lo = 0 when two_terms is False."""
    mx = np.max(np.abs(M), axis=1)
    s = round_fp32(np.where(mx > 0, mx / 448.0, 1.0))
    x = M * (1.0 / s)[:, None]
    hi = round_e4m3(round_fp32(x))
    lo = round_e4m3(round_fp32(x - hi)) if two_terms else np.zeros_like(hi)
    return s, hi, lo


def round_fp16(x: np.ndarray) -> np.ndarray:
    """IEEE binary16 value of each entry, nearest with ties to even: 11
    significant bits for |x| >= 2^-14, the fixed quantum 2^-24 below
    (subnormals); saturating at the largest finite value 65504."""
    x = np.asarray(x, dtype=np.float64)
    normal = round_to_bits(x, 11)
    sub = np.rint(x / 2.0 ** -24) * 2.0 ** -24
    out = np.where(np.abs(x) >= 2.0 ** -14, normal, sub)
    return np.clip(out, -65504.0, 65504.0)


def pow2_scale(mx: np.ndarray, top: int) -> np.ndarray:
    """2^k with mx / 2^k in [2^(top-1), 2^top) (1 where mx = 0); k kept in
    float32's normal exponent range [-126, 127]."""
    mx = np.asarray(mx, dtype=np.float64)
    _, e = np.frexp(mx)                       # mx = m 2^e, 0.5 <= m < 1
    k = np.clip(e - top, -126, 127)
    return np.where(mx > 0, np.ldexp(1.0, k), 1.0)


def quantize_rows_fp16(M: np.ndarray):
    """Per-row FP16 storage with power-of-two scales: s_p = 2^k with
    max_q |M_pq| / s_p in [2^14, 2^15); Q = fp16(M / s) (the scaling exact, one
    rounding).  Returns (s, Q) with M ~ s Q."""
    s = pow2_scale(np.max(np.abs(M), axis=1), 15)
    return s, round_fp16(M / s[:, None])


def quantize_cols_fp16(F: np.ndarray):
    """FP16 right-hand sides [B][n] with power-of-two column scales: t_j = 2^k
    with max_p |F_jp| / t_j in [2^11, 2^12); R = fp16(F / t).  Returns (t, R)."""
    t = pow2_scale(np.max(np.abs(F), axis=1), 12)
    return t, round_fp16(F / t[:, None])


def quantize_fp16_correction(M: np.ndarray):
    """The FP16 store with an e4m3 correction term: (s, Q) = quantize_rows_fp16(M);
    D = M - s Q (exact); (c, C) the per-row e4m3 quantisation of D as in
    quantize_rows_e4m3.  Returns (s, Q, c, C) with M ~ s Q + c C."""
    s, Q = quantize_rows_fp16(M)
    c, C, _ = quantize_rows_e4m3(M - s[:, None] * Q, False)
    return s, Q, c, C


def quantize_bf16_correction(M: np.ndarray):
    """The BF16 store with an e4m3 correction term, written out: Q = bf16(M);
    D = M - Q (exact in FP64: Q holds the leading bits of M); per-row scale
    s_p = float32(max_q |D_pq| / 448) (1 for a zero row); C = e4m3(float32(D / s)).
    Returns (Q, s, C) with M ~ Q + s C."""
    Q = round_bf16(M)
    s, C, _ = quantize_rows_e4m3(M - Q, False)
    return Q, s, C
