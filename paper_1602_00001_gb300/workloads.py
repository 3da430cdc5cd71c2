"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method itself: it only draws node
permittivity fields and charge densities with numpy's seeded generator, and
evaluates the closed-form source and solution of the paper's worked example
(Eqs. 4-5) as inputs.  The
node grid follows Eq. (2): ``nx`` nodes along x (index j, fastest), ``ny``
along y (index i), spacing ``h`` in both directions, boundary nodes included.
Interior arrays are returned in the order of Fig. 3 restricted to the
interior: node (i, j), 1 <= i <= ny-2, 1 <= j <= nx-2 (0-based), flattened
with j fastest.

The shapes follow the paper's workloads (Eq. 4 on [0,1]^2 grids up to 81^2,
Fig. 3's 3x5 grid) widened to the sizes the GPU path is measured at.  No
public dataset exists for this method; everything is synthetic.
"""
from __future__ import annotations

import numpy as np


def node_coords(nx: int, ny: int, h: float):
    """Node coordinates x_j = h*j, y_i = h*i (0-based form of Eq. 2)."""
    x = h * np.arange(nx, dtype=np.float64)
    y = h * np.arange(ny, dtype=np.float64)
    return np.meshgrid(x, y)  # each [ny][nx]


def example_source(x, y):
    """The worked example's right side (Eq. 4) at node coordinates x, y: an
    input, like the seeded fields below."""
    return (12 * x ** 2 - 6 * x) * (y ** 3 - y ** 2) + (x ** 4 - x ** 3) * (6 * y - 2)


def example_exact(x, y):
    """The worked example's exact solution (Eq. 5) at node coordinates x, y:
    the reference its discrete solutions are measured against."""
    return (x ** 4 - x ** 3) * (y ** 3 - y ** 2)


def eps_uniform(nx: int, ny: int) -> np.ndarray:
    """Constant permittivity eps = 1 (the case of Eq. 2 and Fig. 3)."""
    return np.ones((ny, nx), dtype=np.float64)


def eps_fourier(nx: int, ny: int, h: float, seed: int, modes: int = 8,
                amp: float = 0.5) -> np.ndarray:
    """Smooth positive field eps = exp(amp * g).

    g is a sum of ``modes`` x ``modes`` random cosine modes
    a_pq cos(pi p x + phi_pq) cos(pi q y + psi_pq) with a_pq ~ N(0,1)/(1+p^2+q^2),
    normalised to unit standard deviation over the nodes.
    """
    rng = np.random.default_rng(seed)
    X, Y = node_coords(nx, ny, h)
    a = rng.standard_normal((modes, modes))
    phi = rng.uniform(0.0, 2.0 * np.pi, (modes, modes))
    psi = rng.uniform(0.0, 2.0 * np.pi, (modes, modes))
    g = np.zeros_like(X)
    for p in range(modes):
        for q in range(modes):
            g += (a[p, q] / (1.0 + p * p + q * q)
                  * np.cos(np.pi * p * X + phi[p, q]) * np.cos(np.pi * q * Y + psi[p, q]))
    g = (g - g.mean()) / max(g.std(), 1e-300)
    return np.exp(amp * g)


def eps_lognormal(nx: int, ny: int, seed: int, sigma: float = 0.5) -> np.ndarray:
    """Rough positive field eps = exp(sigma * z), z i.i.d. N(0,1) per node."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal((ny, nx)))


def _interior(a: np.ndarray) -> np.ndarray:
    """[..., ny, nx] node array -> [..., (ny-2)*(nx-2)] interior, j fastest."""
    core = a[..., 1:-1, 1:-1]
    return np.ascontiguousarray(core.reshape(core.shape[:-2] + (-1,)))


def gaussian_blobs(nx: int, ny: int, h: float, seed: int, nblobs: int = 4,
                   width: float = 0.05, batch: int = 1) -> np.ndarray:
    """Charge density rho as a sum of ``nblobs`` Gaussian blobs per column.

    Centres uniform in [0.2, 0.8] of each side, width ``width`` (same units as
    h), amplitudes N(0,1).  Returns [batch][n_interior] float64.
    """
    rng = np.random.default_rng(seed)
    X, Y = node_coords(nx, ny, h)
    lx, ly = h * (nx - 1), h * (ny - 1)
    out = np.zeros((batch, ny, nx))
    for c in range(batch):
        cx = rng.uniform(0.2, 0.8, nblobs) * lx
        cy = rng.uniform(0.2, 0.8, nblobs) * ly
        amp = rng.standard_normal(nblobs)
        for k in range(nblobs):
            out[c] += amp[k] * np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2 * width ** 2))
    return _interior(out)


def moving_charges(nx: int, ny: int, h: float, seed: int, steps: int,
                   ncharges: int = 16, width: float = 0.04,
                   path: str = "circle") -> np.ndarray:
    """rho(x, t) of ``ncharges`` Gaussian charges moving over ``steps`` steps.

    ``path='circle'``: each charge runs a circle of random centre, radius,
    phase and angular speed; ``path='line'``: a straight segment between two
    random points.  Column t of the result is the density at time step t.
    Returns [steps][n_interior] float64.
    """
    rng = np.random.default_rng(seed)
    X, Y = node_coords(nx, ny, h)
    lx, ly = h * (nx - 1), h * (ny - 1)
    q = rng.standard_normal(ncharges)
    if path == "circle":
        c0 = rng.uniform(0.35, 0.65, (ncharges, 2))
        rad = rng.uniform(0.05, 0.25, ncharges)
        ph = rng.uniform(0, 2 * np.pi, ncharges)
        om = rng.uniform(0.5, 2.0, ncharges) * 2 * np.pi / max(steps, 1)
    else:
        p0 = rng.uniform(0.2, 0.8, (ncharges, 2))
        p1 = rng.uniform(0.2, 0.8, (ncharges, 2))
    core = np.zeros((steps, ny - 2, nx - 2))
    Xi, Yi = X[1:-1, 1:-1], Y[1:-1, 1:-1]
    for t in range(steps):
        for k in range(ncharges):
            if path == "circle":
                cx = (c0[k, 0] + rad[k] * np.cos(ph[k] + om[k] * t)) * lx
                cy = (c0[k, 1] + rad[k] * np.sin(ph[k] + om[k] * t)) * ly
            else:
                s = t / max(steps - 1, 1)
                cx = ((1 - s) * p0[k, 0] + s * p1[k, 0]) * lx
                cy = ((1 - s) * p0[k, 1] + s * p1[k, 1]) * ly
            core[t] += q[k] * np.exp(-((Xi - cx) ** 2 + (Yi - cy) ** 2) / (2 * width ** 2))
    return core.reshape(steps, -1)


def random_interior(nx: int, ny: int, seed: int, batch: int = 1) -> np.ndarray:
    """Rough i.i.d. N(0,1) interior vectors (worst case for accuracy)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, (ny - 2) * (nx - 2)))


def batched_problem_set(seed: int, nprob: int = 64, sides=(32, 48, 64, 96, 128),
                        bmax: int = 64):
    """Uneven problem list: side n uniform over ``sides``, lognormal eps
    (sigma 0.5), ragged RHS count uniform over 1..bmax.  Returns a list of
    (side, eps[side][side], rho[B][n_interior]) with h = 1/(side-1)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nprob):
        side = int(rng.choice(sides))
        B = int(rng.integers(1, bmax + 1))
        sub = int(rng.integers(0, 2**31 - 1))
        h = 1.0 / (side - 1)
        eps = eps_lognormal(side, side, sub, 0.5)
        rho = gaussian_blobs(side, side, h, sub + 1, batch=B)
        out.append((side, eps, rho))
    return out
