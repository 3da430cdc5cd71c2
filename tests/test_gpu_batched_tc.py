"""Batched plans on the tensor cores: FP32 stores contracted as TF32 in the
grouped tcgen05 launch, the column-tile width per problem (the knob the
autotuner sets), and the plan's report of the shapes it launches.

* One TF32 apply (no sweep) of an FP32 store equals the FP64 product of the
  oracle's FP32 roundings of the inverse and of the right-hand side within
  TF32's reading of both operands (10 explicit mantissa bits each: 2^-9 of
  |A||x| in all), and is measurably coarser than the FP32 SIMT tiles' product
  (which holds 1e-5 of |A||x|): the tensor-core path is the one that ran.
* Refined, TF32 problems of the 64-grid configuration's sizes reach the
  oracle to 1e-6 with two sweeps.
* Column tiles of 32, 64 or 128 change the launched items, not the result
  (bit for bit: the K order of every sum is the same); SIMT tile widths
  16/32/64 likewise."""
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


def _problem(side, B, prec, seed):
    from paper_1602_00001_gb300.binding import Solver
    h = 1.0 / (side - 1)
    eps = W.eps_lognormal(side, side, seed=seed)
    b = O.rhs_from_charge(side, side, h, eps, W.gaussian_blobs(side, side, h, seed + 1, batch=B))
    return Solver(side, side, h, eps, prec), eps, b


@pytest.mark.parametrize("tc", [1, 0])
def test_fp32_one_apply_bound(tc):
    from paper_1602_00001_gb300.binding import BatchPlan
    side, B = 37, 45
    s, eps, b = _problem(side, B, "fp32", 5)
    s.set_tuning(batch_tc=tc)
    bd = torch.from_numpy(b).cuda()
    u = torch.full_like(bd, float("nan"))
    plan = BatchPlan([s], [bd], [u])
    info = plan.info()
    assert info["tf32_problems"] == tc and (info["tc_items"] > 0) == (tc == 1)
    plan.run(sweeps=0, use_graph=False)
    torch.cuda.synchronize()
    A = O.round_fp32(O.interior_inverse(side, side, eps))
    x = O.round_fp32(b)
    ref = x @ A.T
    mag = np.abs(x) @ np.abs(A).T
    rel = np.abs(u.cpu().numpy() - ref) / mag
    if tc:
        assert np.max(rel) <= 2.0 ** -9 and np.max(rel) > 2.0 ** -16, float(np.max(rel))
    else:
        assert np.max(rel) <= 1e-5, float(np.max(rel))
    plan.close()
    s.close()


def test_tf32_refined_config_sizes():
    from paper_1602_00001_gb300.binding import BatchPlan
    sides, Bs = [128, 96, 64, 48, 32], [64, 17, 1, 40, 9]
    solvers, bs, us, refs = [], [], [], []
    for k, (side, B) in enumerate(zip(sides, Bs)):
        s, eps, b = _problem(side, B, "fp32" if k != 3 else "bf16", 30 + k)
        solvers.append(s)
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.empty_like(bs[-1]))
        cols = [0, B - 1]
        refs.append((cols, O.solve(side, side, eps, b[cols], route="band")))
    caps = [2 if s.precision == "fp32" else 6 for s in solvers]
    plan = BatchPlan(solvers, bs, us, sweeps_per_problem=caps)
    assert plan.info()["tf32_problems"] == 4
    plan.run(sweeps=6, use_graph=False)
    torch.cuda.synchronize()
    for u, (cols, r) in zip(us, refs):
        assert O.rel_error_eq6(u[cols].cpu().numpy(), r) < 1e-6
    plan.close()


def test_column_tile_knob_changes_items_not_results():
    from paper_1602_00001_gb300.binding import BatchPlan
    probs = [_problem(41, 70, "fp32", 50), _problem(29, 33, "bf16", 52)]
    outs = {}
    for bn in (32, 64, 128):
        solvers, bs, us = [], [], []
        for s, _, b in probs:
            s.set_tuning(batch_bn=bn)
            solvers.append(s)
            bs.append(torch.from_numpy(b).cuda())
            us.append(torch.empty_like(bs[-1]))
        plan = BatchPlan(solvers, bs, us)
        info = plan.info()
        n0, n1 = solvers[0].n, solvers[1].n
        expect = ((n0 + 127) // 128) * ((70 + bn - 1) // bn) + ((n1 + 127) // 128) * ((33 + bn - 1) // bn)
        assert info["tc_items_bn"][bn] == expect and info["tc_items"] == expect
        assert info["apply_launches"] == 1 and info["simt_items"] == 0
        plan.run(sweeps=3, use_graph=False)
        torch.cuda.synchronize()
        outs[bn] = [u.clone() for u in us]
        plan.close()
    for bn in (64, 128):
        for a, c in zip(outs[32], outs[bn]):
            assert torch.equal(a, c), bn
    for s, _, _ in probs:
        s.close()


def test_simt_tile_knob():
    from paper_1602_00001_gb300.binding import BatchPlan
    s, eps, b = _problem(33, 50, "fp32", 60)
    s.set_tuning(batch_tc=0)
    bd = torch.from_numpy(b).cuda()
    outs = []
    for tn in (16, 32, 64):
        s.set_tuning(batch_tn=tn)
        u = torch.empty_like(bd)
        plan = BatchPlan([s], [bd], [u])
        info = plan.info()
        assert info["simt_problems_tn"][tn] == 1 and info["tc_items"] == 0
        plan.run(sweeps=2, use_graph=False)
        torch.cuda.synchronize()
        outs.append(u.clone())
        plan.close()
    for o in outs[1:]:
        assert float((o - outs[0]).abs().max()) <= 1e-12 * float(outs[0].abs().max())
    ref = O.solve(33, 33, eps, b[[0, 49]], route="band")
    assert O.rel_error_eq6(outs[0][[0, 49]].cpu().numpy(), ref) < 1e-6
    s.close()
