"""Adjoint kernels: dLoss/db and dLoss/deps of Loss = 0.5 ||u - u_t||^2,
u = L(eps)^-1 b, against the oracle's gradient and FP64 central finite
differences (128 x 128 nodes, 126^2 unknowns, lognormal eps, B = 32)."""
import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 128
B = 32


@pytest.fixture(scope="module")
def case():
    from paper_1602_00001_gb300 import build, binding
    build.build()
    binding.load_library()
    h = 1.0 / (N - 1)
    eps = W.eps_lognormal(N, N, seed=4)
    rho = W.gaussian_blobs(N, N, h, seed=40, batch=B)
    b = O.rhs_from_charge(N, N, h, eps, rho)
    rho_t = W.gaussian_blobs(N, N, h, seed=41, batch=B)
    ut = O.solve(N, N, eps, O.rhs_from_charge(N, N, h, eps, rho_t), route="band")
    return h, eps, b, ut


def _grads(solver, b, ut, sweeps):
    bd = torch.from_numpy(b).cuda()
    u = solver.apply(bd, sweeps=sweeps)
    g = u - torch.from_numpy(ut).cuda()
    db, deps = solver.backward(g, u, bd, sweeps=sweeps)
    return u.cpu().numpy(), db.cpu().numpy(), deps.cpu().numpy()


def test_backward_matches_oracle_gradient(case):
    from paper_1602_00001_gb300.binding import Solver
    h, eps, b, ut = case
    u_o = O.solve(N, N, eps, b, route="band")
    _, db_o, deps_o = O.adjoint_gradients(N, N, eps, b, u_o - ut)
    for prec, sweeps, tol in (("fp64", 0, 1e-11), ("bf16", 5, 1e-6)):
        s = Solver(N, N, h, eps, prec)
        u, db, deps = _grads(s, b, ut, sweeps)
        assert O.rel_error_eq6(u, u_o) < tol
        assert np.max(np.abs(db - db_o)) <= tol * np.max(np.abs(db_o)), prec
        assert np.max(np.abs(deps - deps_o)) <= tol * np.max(np.abs(deps_o)), prec
        s.close()


def test_backward_against_central_differences(case):
    """FP64 central differences (relative step 1e-6) of the GPU FP64 solve on
    50 random eps entries and 50 b entries, against the refined BF16
    backward, to 1e-5."""
    from paper_1602_00001_gb300.binding import Solver
    h, eps, b, ut = case
    s = Solver(N, N, h, eps, "bf16")
    _, db, deps = _grads(s, b, ut, 6)
    s.close()
    bd = torch.from_numpy(b).cuda()
    utd = torch.from_numpy(ut).cuda()

    def loss(solver, bb):
        u = solver.apply(bb)
        return 0.5 * float(((u - utd) ** 2).sum())

    rng = np.random.default_rng(3)
    scale_e = np.max(np.abs(deps))
    nodes = rng.choice(N * N, 50, replace=False)
    for k in nodes:
        i, j = divmod(int(k), N)
        st = 1e-6 * eps[i, j]
        vals = []
        for sgn in (1, -1):
            e2 = eps.copy()
            e2[i, j] += sgn * st
            sp = Solver(N, N, h, e2, "fp64")
            vals.append(loss(sp, bd))
            sp.close()
        fd = (vals[0] - vals[1]) / (2 * st)
        assert abs(fd - deps[i, j]) <= 1e-5 * scale_e, (i, j, fd, deps[i, j])
    s64 = Solver(N, N, h, eps, "fp64")
    scale_b = np.max(np.abs(db))
    for _ in range(50):
        c, p = int(rng.integers(B)), int(rng.integers(s64.n))
        st = 1e-6 * np.max(np.abs(b[c]))
        bp, bm = bd.clone(), bd.clone()
        bp[c, p] += st
        bm[c, p] -= st
        fd = (loss(s64, bp) - loss(s64, bm)) / (2 * st)
        assert abs(fd - db[c, p]) <= 1e-5 * scale_b, (c, p, fd, db[c, p])


def test_autograd_function(case):
    """torch.autograd through the C ABI: gradients equal the direct backward."""
    from paper_1602_00001_gb300.binding import Solver, pide_apply_autograd
    h, eps, b, ut = case
    s = Solver(N, N, h, eps, "bf16")
    bd = torch.from_numpy(b).cuda().requires_grad_(True)
    et = torch.from_numpy(eps).cuda().requires_grad_(True)
    u = pide_apply_autograd(bd, et, s, 5)
    loss = 0.5 * ((u - torch.from_numpy(ut).cuda()) ** 2).sum()
    loss.backward()
    _, db, deps = _grads(s, b, ut, 5)
    assert np.max(np.abs(bd.grad.cpu().numpy() - db)) <= 1e-12 * np.max(np.abs(db))
    assert np.max(np.abs(et.grad.cpu().numpy() - deps)) <= 1e-12 * np.max(np.abs(deps))
