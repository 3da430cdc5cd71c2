"""Batched apply over uneven grids with ragged column counts (FP32 and BF16
stores), against the oracle per problem."""
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


def _run(sides, Bs, precs, sweeps, seed):
    from paper_1602_00001_gb300.binding import Solver, apply_batched
    solvers, bs, us, refs = [], [], [], []
    for k, (side, B, prec) in enumerate(zip(sides, Bs, precs)):
        h = 1.0 / (side - 1)
        eps = W.eps_lognormal(side, side, seed=seed + k)
        rho = W.gaussian_blobs(side, side, h, seed=seed + 100 + k, batch=B)
        b = O.rhs_from_charge(side, side, h, eps, rho)
        solvers.append(Solver(side, side, h, eps, prec))
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.empty_like(bs[-1]))
        refs.append(O.solve(side, side, eps, b))
    apply_batched(solvers, bs, us, sweeps=sweeps)
    torch.cuda.synchronize()
    return [O.rel_error_eq6(u.cpu().numpy(), r) for u, r in zip(us, refs)]


def test_batched_small_uneven():
    errs = _run([12, 20, 33, 9, 27, 16], [1, 5, 17, 64, 3, 40],
                ["fp32", "bf16", "fp32", "bf16", "bf16", "fp32"], 8, seed=1)
    assert max(errs) < 1e-6, errs


def test_batched_config_sizes():
    """Grids with the sizes of the 64-grid configuration (sides 32..128)."""
    rng = np.random.default_rng(3)
    sides = [int(x) for x in rng.choice([32, 48, 64, 96, 128], 8)]
    Bs = [int(x) for x in rng.integers(1, 65, 8)]
    precs = ["bf16" if k % 2 else "fp32" for k in range(8)]
    errs = _run(sides, Bs, precs, 8, seed=10)
    assert max(errs) < 1e-6, errs


def test_batch_plan_graph_replay():
    """A plan replayed from its captured CUDA graph gives the same result as
    direct launches, run after run, and matches the oracle."""
    from paper_1602_00001_gb300.binding import Solver, BatchPlan
    sides, Bs = [14, 26, 40, 19], [3, 64, 9, 33]
    solvers, bs, us, refs = [], [], [], []
    for k, (side, B) in enumerate(zip(sides, Bs)):
        h = 1.0 / (side - 1)
        eps = W.eps_lognormal(side, side, seed=70 + k)
        b = O.rhs_from_charge(side, side, h, eps, W.gaussian_blobs(side, side, h, 80 + k, batch=B))
        solvers.append(Solver(side, side, h, eps, "bf16" if k % 2 else "fp32"))
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.zeros_like(bs[-1]))
        refs.append(O.solve(side, side, eps, b))
    plan = BatchPlan(solvers, bs, us)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.run(sweeps=8, use_graph=False, stream=stream)
    stream.synchronize()
    direct = [u.clone() for u in us]
    for _ in range(2):
        for u in us:
            u.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            plan.run(sweeps=8, use_graph=True, stream=stream)
        stream.synchronize()
        for u, d in zip(us, direct):
            assert torch.equal(u, d)
    for u, r in zip(us, refs):
        assert O.rel_error_eq6(u.cpu().numpy(), r) < 1e-6
    plan.close()


def test_batched_rejects_fp64_store():
    from paper_1602_00001_gb300.binding import Solver, BatchPlan, PideError
    s = Solver(10, 10, 1 / 9, None, "fp64")
    b = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(PideError):
        BatchPlan([s], [b], [torch.empty_like(b)])


def test_batch_plan_per_problem_sweeps():
    """FP32 problems capped at 2 sweeps, BF16 at 8, in one plan."""
    from paper_1602_00001_gb300.binding import Solver, BatchPlan
    sides, Bs = [30, 45, 22, 37], [7, 64, 1, 20]
    solvers, bs, us, refs, caps = [], [], [], [], []
    for k, (side, B) in enumerate(zip(sides, Bs)):
        h = 1.0 / (side - 1)
        eps = W.eps_lognormal(side, side, seed=90 + k)
        b = O.rhs_from_charge(side, side, h, eps, W.gaussian_blobs(side, side, h, 95 + k, batch=B))
        prec = "fp32" if k % 2 == 0 else "bf16"
        solvers.append(Solver(side, side, h, eps, prec))
        caps.append(2 if prec == "fp32" else 8)
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.zeros_like(bs[-1]))
        refs.append(O.solve(side, side, eps, b))
    plan = BatchPlan(solvers, bs, us, sweeps_per_problem=caps)
    plan.run(sweeps=8, use_graph=False)
    torch.cuda.synchronize()
    for u, r in zip(us, refs):
        assert O.rel_error_eq6(u.cpu().numpy(), r) < 1e-6
    plan.close()
