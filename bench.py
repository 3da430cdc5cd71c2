"""Benchmark: refined low-precision dense-inverse apply, u = L_eps^-1 b, on a
200 x 200 node grid (198^2 = 39204 unknowns) with B = 1024 right-hand sides.

One step = one refined apply of the whole batch: right-hand-side prep, the
first tensor-core apply and k refinement sweeps (stencil residual + apply),
inputs resident in HBM.  The store is chosen by the library from the
refinement's measured contraction (pide_setup_auto with its built-in probes,
target 0.5e-6; on GB300 this picks FP16 with power-of-two row scales plus an
e4m3 correction term added in the first apply); --precision forces BF16,
BF16 + e4m3, FP16, FP16 + e4m3, FP8 hi+lo or FP32.  The e2e figure streams
steps from pinned host memory through pide_solve_stream (copies in and out
inside the timed region).  k is the smallest sweep count whose Eq. (6) error
against the plain FP64 GPU apply is <= 0.5e-6 on sampled columns (checked
against the FP64 oracle on four columns in the CPU-baseline leg); the sweep
count the library measured is reported beside it.  The metric is
right-hand-side solves per second, whole job (all ranks).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload batched | adjoint | 3d | formats
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NODES = 200                  # grid nodes per side (Eq. 2), 198^2 interior unknowns
BATCH = 1024                 # right-hand sides per step
PRECISION = "auto"
METRIC = "RHS solves/s at 198^2 grid, B=1 and 1024, refined BF16/FP8 vs FP64 apply @1e-6"
UNIT = "RHS solves/s"
TARGET_ERR = 0.5e-6          # calibration target (the bar is 1e-6)
WORKLOAD = "198^2 interior (200x200 nodes), Fourier-field eps, 16 moving charges, B=1024"


# DRAM traffic (read + write) of one launch of the GEMM at this workload, from a
# one-pass ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of the SM-pair
# GEMM launches of a timed step); valid only for the kernel source it was taken on
# (sha1 of csrc/gemm_tc2.cu + csrc/common.cuh), and reported as a stored figure.
# Average over the FP16 launches of two timed steps (first apply 5.02-5.60 GB, the
# refinement apply 7.97-8.26 GB); the e4m3 correction GEMM (2.51 GB) is reported on its own.
GEMM_TRAFFIC = {"sha1": "33ed1ddd706b9dc4cad88dca1026be7394ebb618", "bytes": 6.71e9,
                "precision": "fp16_fp8", "batch": 1024, "nodes": 200, "sweeps": 1,
                "corr_mask": 1, "corr_bytes": 2.51e9, "a_hint": 2,
                "source": "stored ncu capture of this kernel source (dram__bytes_read.sum + "
                          "dram__bytes_write.sum, one pass, NVTX-selected timed steps)"}


def gemm_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("gemm_tc2.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1602_00001_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi needs a moment before its first line: wait for it, then
            # keep only the samples taken inside the timed region
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.02)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, dist=None) -> float:
    """Max over ranks of a per-rank time (gloo: CPU tensor; nccl: CUDA tensor)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, per_rank_batch: int, steps: int, ms_total_max: float) -> float:
    """Right-hand sides solved by all ranks per second of the slowest rank."""
    return world * per_rank_batch * steps / (ms_total_max / 1e3)


# BLAS / OpenMP thread counts of the host processes that time the oracle
THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _cpu_band_worker(nodes, seed, cols, col0, reps, warm, barrier, out_q):
    """One host process: the oracle's band-LU factorisation of the workload's
    operator (untimed, setup), then `reps` timed band solves of `cols` of its
    columns, started together with the other processes."""
    from oracle import pide_oracle as O
    from paper_1602_00001_gb300 import workloads as W
    h = 1.0 / (nodes - 1)
    eps = W.eps_fourier(nodes, nodes, h, seed=seed)
    rho = W.moving_charges(nodes, nodes, h, seed=seed, steps=BATCH)[col0:col0 + cols]
    b = O.rhs_from_charge(nodes, nodes, h, eps, rho)
    fac = O.BandSolver(nodes, nodes, eps)
    for _ in range(warm):
        fac.solve(b)
    barrier.wait()
    t = time.perf_counter()
    u = None
    for _ in range(max(reps, 1)):
        u = fac.solve(b)
    out_q.put((col0, time.perf_counter() - t, u if col0 == 0 else None))


def _cpu_dense_worker(nodes, seed, out_q):
    """One host process: the oracle's dense FP64 inverse of a grid that fits
    host memory (formed untimed), then its dense apply (numpy/BLAS with the
    thread count of this process's environment) at B = 1 and B = 64."""
    from oracle import pide_oracle as O
    from paper_1602_00001_gb300 import workloads as W
    h = 1.0 / (nodes - 1)
    eps = W.eps_fourier(nodes, nodes, h, seed=seed)
    Linv = O.interior_inverse(nodes, nodes, eps, route="band")
    b = O.rhs_from_charge(nodes, nodes, h, eps,
                          W.moving_charges(nodes, nodes, h, seed=seed, steps=64))
    out = {}
    for B in (1, 64):
        O.apply_inverse(Linv, b[:B])
        reps, t = 0, time.perf_counter()
        while time.perf_counter() - t < 1.0 or reps < 3:
            O.apply_inverse(Linv, b[:B])
            reps += 1
        out[B] = B * reps / (time.perf_counter() - t)
    out_q.put(out)


def _spawn_with_threads(threads, target, args_list, timeout=900):
    """Run target(*args, barrier, queue) (or target(*args, queue)) in fresh
    spawned processes whose BLAS/OpenMP pools have `threads` threads; returns
    the queued results."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    for k in THREAD_VARS:
        os.environ[k] = str(threads)
    try:
        q = ctx.Queue()
        barrier = ctx.Barrier(len(args_list)) if target is _cpu_band_worker else None
        procs = []
        for a in args_list:
            extra = (barrier, q) if barrier is not None else (q,)
            procs.append(ctx.Process(target=target, args=(*a, *extra)))
        for p in procs:
            p.start()
        res = [q.get(timeout=timeout) for _ in procs]
        for p in procs:
            p.join(timeout=60)
        return res
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_band_rate(nodes, seed, procs, cols, reps, warm=0):
    """Oracle band-LU solves/s of the workload on `procs` single-threaded host
    processes, `cols` columns each: (rate, max seconds, solution of columns 0..cols-1)."""
    res = _spawn_with_threads(1, _cpu_band_worker,
                              [(nodes, seed, cols, i * cols, reps, warm) for i in range(procs)])
    tmax = max(r[1] for r in res)
    u0 = next(r[2] for r in res if r[0] == 0)
    return procs * cols * max(reps, 1) / tmax, tmax, u0


def cpu_baseline_leg(nodes, seed, cores, cols=4):
    """The oracle on the host cores: the workload's band-LU solve on one core
    and on every core (one process per core), and the dense FP64 apply of a
    100 x 100 node grid (98^2 unknowns, inverse 0.74 GB) at B = 1 and 64 with
    one BLAS thread and with all of them."""
    t0 = time.perf_counter()
    r1, t1, u0 = cpu_band_rate(nodes, seed, 1, cols, 1)
    rall, tall, _ = cpu_band_rate(nodes, seed, cores, cols, 1)
    d1 = _spawn_with_threads(1, _cpu_dense_worker, [(100, seed)])[0]
    dall = _spawn_with_threads(cores, _cpu_dense_worker, [(100, seed)])[0]
    return {
        "value": rall, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": (f"numpy band-LU solve of {cols} of the {BATCH} columns per process, one "
                   f"single-threaded process per host core ({cores}), started together "
                   f"({tall:.2f} s); factorisation untimed (setup)"),
        "host_cores": os.cpu_count(),
        "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                        "sample": f"{cols} columns, one process ({t1:.2f} s)"},
        "dense_apply_98sq": {
            "unit": UNIT, "note": "oracle's dense FP64 inverse of a 100x100 node grid "
                                  "(9604 unknowns) applied with numpy (BLAS); the 198^2 "
                                  "inverse (12.3 GB) is not formed on the host",
            "b1": {"single_thread": d1[1], "all_threads": dall[1]},
            "b64": {"single_thread": d1[64], "all_threads": dall[64]},
            "threads": cores},
        "leg_seconds": time.perf_counter() - t0,
    }, u0


def reference_arm(args):
    """--impl reference: the FP64 oracle, as it stands, on the host cores (one
    single-threaded band-LU process per core, each solving its own 4 columns of
    the workload per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cols = 4
    cores = max(1, min(os.cpu_count() or 1, BATCH // cols))
    value, tmax, _ = cpu_band_rate(NODES, 5, cores, cols, args.steps, args.warmup)
    dt = tmax / max(args.steps, 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": cols * cores, "grid": "200x200",
                   "sample": f"{cols} columns per process per step, {cores} processes"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"numpy band-LU forward/back substitution, {cols} of the "
                                   f"1024 columns per process and step, {cores} single-threaded "
                                   "processes started together; factorisation untimed (setup)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _evt_time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    z.record()
    torch.cuda.synchronize()
    return a.elapsed_time(z) / reps


def batched_workload(args):
    """64 independent grids (side uniform over {32,48,64,96,128}, lognormal eps
    sigma 0.5), ragged B_k uniform over 1..64, FP32 and BF16 stores alternating:
    one plan (one launch per phase, replayed from a CUDA graph) against a loop
    of per-problem pide_apply calls with the same sweep counts.  Each problem's
    sweep count is calibrated like the headline's, on the plan's own
    arithmetic: the smallest count whose Eq. (6) error against that problem's
    FP64 GPU apply is <= TARGET_ERR."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_00001_gb300 import workloads as W
    from paper_1602_00001_gb300.binding import Solver, BatchPlan
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    probs = W.batched_problem_set(seed=3, nprob=64)
    solvers, bs, us, refs = [], [], [], []
    for k, (side, eps, rho) in enumerate(probs):
        h = 1.0 / (side - 1)
        sv = Solver(side, side, h, eps, "fp32" if k % 2 == 0 else "bf16")
        bd = sv.rhs_from_charge(torch.from_numpy(rho).cuda())
        s64 = Solver(side, side, h, eps, "fp64")
        refs.append(s64.apply(bd))
        s64.close()
        solvers.append(sv)
        bs.append(bd)
        us.append(torch.empty_like(bd))
    total_rhs = sum(b.shape[0] for b in bs)

    def rel_err(uu, ref):
        return float(((uu - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max())
    # the autotuner times the plan's knobs (tensor-core column tile, FP32 on the
    # tensor cores or the SIMT tiles) on one problem of each (precision, n, B)
    # bucket with two sweeps, outside the timed region; plans are built from
    # its cache
    from paper_1602_00001_gb300 import autotune as AT
    cache = AT.TuneCache(os.path.join(ROOT, "_build", "pide_tune_bench.json"))
    t_tune = time.perf_counter()
    tuned = {}
    for sv, b, u in zip(solvers, bs, us):
        key = AT.batch_key_for(sv.n, b.shape[0], sv.precision)
        if key not in tuned:
            tuned[key] = AT.tune_batch(sv, b, u, sweeps=2, cache=cache, save=False)[0]
    t_tune = time.perf_counter() - t_tune
    nprob = len(solvers)
    if args.sweeps >= 0:
        # an FP32 store converges in far fewer sweeps than a BF16 one: a forced
        # count is capped at 2 for it
        caps = [min(2, args.sweeps) if sv.precision == "fp32" else args.sweeps for sv in solvers]
        calib = None
    else:
        # calibrated through a plan of the same shapes (its FP32 problems run on
        # the TF32 tensor cores, unlike pide_apply's FP32 SIMT apply): run it
        # with k = 0, 1, ... sweeps and give each problem the first k at which
        # its Eq. 6 error against its FP64 GPU apply is <= TARGET_ERR
        probe = BatchPlan(solvers, bs, us, sweeps_per_problem=[8] * nprob, tune_cache=cache)
        caps, calib = [None] * nprob, [None] * nprob
        for kk in range(0, 9):
            probe.run(kk, use_graph=False)
            torch.cuda.synchronize()
            for q in range(nprob):
                if caps[q] is None:
                    e = rel_err(us[q], refs[q])
                    if e <= TARGET_ERR or kk == 8:
                        caps[q], calib[q] = kk, e
            if all(c is not None for c in caps):
                break
        probe.close()
    sweeps = max(caps)
    plan = BatchPlan(solvers, bs, us, sweeps_per_problem=caps, tune_cache=cache)
    pinfo = plan.info()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan.run(sweeps, use_graph=True, stream=st)
    st.synchronize()
    # every problem of the plan's result against its FP64 GPU apply
    errs = [rel_err(u, ref) for u, ref in zip(us, refs)]
    del refs
    with torch.cuda.stream(st):
        torch.cuda.nvtx.range_push("timed_steps")
        ms_batched = _evt_time(lambda: plan.run(sweeps, use_graph=True, stream=st), args.steps)
        torch.cuda.nvtx.range_pop()

    def loop():
        for sv, b, u, kc in zip(solvers, bs, us, caps):
            sv.apply(b, u, sweeps=kc)
    ms_loop = _evt_time(loop, max(3, args.steps // 4))
    launches = 1 + (1 + sweeps) * pinfo["apply_launches"] + sweeps
    hist = {}
    for sv, kc in zip(solvers, caps):
        d = hist.setdefault(sv.precision, {})
        d[str(kc)] = d.get(str(kc), 0) + 1
    line = {"metric": "RHS solves/s, 64 uneven grids (batched)", "value": total_rhs / (ms_batched * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": ms_batched,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32+bf16",
            "data": "synthetic",
            "config": {"workload": "64 grids, side in {32,48,64,96,128}, lognormal eps, B_k in 1..64",
                       "total_rhs": total_rhs,
                       "sweeps": "per problem, calibrated to Eq. 6 error <= %g vs its FP64 GPU apply"
                                 % TARGET_ERR if args.sweeps < 0 else f"forced {args.sweeps}",
                       "sweep_counts": hist, "sizes": [int(p[0]) for p in probs]},
            "per_problem_loop": {"ms_per_step": ms_loop, "value": total_rhs / (ms_loop * 1e-3)},
            "speedup_vs_loop": ms_loop / ms_batched, "gpu_launches_per_step": launches,
            "plan": pinfo, "tuning": {"chosen": tuned, "seconds": t_tune,
                                      "source": "autotune.tune_batch per (precision, n, B) bucket"},
            "roofline": batched_roofline(solvers, bs, caps, ms_batched),
            "accuracy": {"max_rel_err_eq6_vs_fp64_gpu_all_problems": max(errs),
                         "calibration_max_err": max(calib) if calib else None}}
    print(json.dumps(line))
    return 0


def batched_roofline(solvers, bs, caps, ms):
    """HBM view of a batched step.  Per problem (n unknowns, B columns, store
    entries of e = 2 (BF16) or 4 (FP32) bytes) and per phase it runs (1 + cap):
    the stored inverse n^2 e, the right-hand side R (n B e: written by the vector
    pass, read by the apply), u (8 n B written by the first apply, read and
    written by each later one), b (8 n B read by every vector pass) and u again
    (8 n B read by each residual).  The fraction is taken on all of it; the
    inverse bytes alone are reported beside it."""
    pk, kind = peaks()
    inv, total = 0.0, 0.0
    for sv, b, cap in zip(solvers, bs, caps):
        esz = 4 if sv.precision == "fp32" else 2
        n, B, ph = sv.n, b.shape[0], 1 + cap
        inv += ph * n * n * esz
        total += ph * (n * n * esz + 2 * n * B * esz + 8 * n * B) + cap * (16 + 8) * n * B
        total += 8 * n * B                            # the first vector pass's read of b
    gbs = total / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / pk["hbm_gbs"], "traffic": None,
            "algorithmic_bytes_per_step": total, "inverse_bytes_per_step": inv,
            "inverse_only_frac": inv / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
            "note": "all algorithmic bytes of the step (inverse, R, u, b); FP32 problems run "
                    "on the TF32 tensor cores unless their knob keeps the SIMT tiles"}


def adjoint_workload(args):
    """128 x 128 nodes (126^2 unknowns), lognormal eps, B = 32: forward refined
    apply plus the backward (adjoint solve, dLoss/db, dLoss/deps) per step."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_00001_gb300 import workloads as W
    from paper_1602_00001_gb300.binding import Solver
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    N, B = 128, 32
    h = 1.0 / (N - 1)
    eps = W.eps_lognormal(N, N, seed=4)
    prec = args.precision or "fp16_fp8"
    s = Solver(N, N, h, eps, prec)
    b = s.rhs_from_charge(torch.from_numpy(W.gaussian_blobs(N, N, h, seed=40, batch=B)).cuda())
    ut = s.apply(s.rhs_from_charge(torch.from_numpy(W.gaussian_blobs(N, N, h, seed=41, batch=B)).cuda()), sweeps=6)
    sweeps = args.sweeps if args.sweeps >= 0 else {"bf16_fp8": 2, "fp16_fp8": 1, "fp16": 2}.get(prec, 5)
    # bytes each solve streams: the BF16 inverse every apply, the e4m3 correction
    # term (with its row scales) in the applies the correction mask selects
    n, ld = s.n, s.info().ld
    hi_bytes = 2 * n * ld if prec in ("bf16", "bf16_fp8", "fp16", "fp16_fp8") else s.info().store_bytes
    mask = s.get_tuning()["corr_mask"] if prec.endswith("_fp8") else 0
    n_corr = sum((mask >> k) & 1 for k in range(sweeps + 1))
    solve_bytes = (1 + sweeps) * hi_bytes + n_corr * (n * ld + 4 * n)

    def step():
        u = s.apply(b, sweeps=sweeps)
        return s.backward(u - ut, u, b, sweeps=sweeps)
    db, deps = step()
    # the same gradients through the plain FP64 GPU path (FP64 inverse, FP64
    # forward and adjoint applies); the tests check that path against the oracle
    s64 = Solver(N, N, h, eps, "fp64")
    u64 = s64.apply(b)
    db_o, deps_o = s64.backward(u64 - ut, u64, b, sweeps=0)
    s64.close()
    err_db = float((db - db_o).abs().max() / db_o.abs().max())
    err_de = float((deps - deps_o).abs().max() / deps_o.abs().max())
    ms = _evt_time(step, args.steps)
    line = {"metric": "forward+backward RHS/s, 126^2 grid, B=32", "value": B / (ms * 1e-3),
            "unit": "RHS/s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
            "data": "synthetic", "config": {"workload": "128x128 nodes, lognormal eps, B=32",
                                            "sweeps": sweeps, "precision": prec},
            "accuracy": {"db_rel_err_vs_fp64_gpu": err_db, "deps_rel_err_vs_fp64_gpu": err_de},
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peaks()[0]["hbm_gbs"],
                         "achieved": 2 * solve_bytes / (ms * 1e-3) / 1e9,
                         "note": "B = 32 is HBM-bound: forward and adjoint solves each stream the "
                                 "BF16 inverse 1 + sweeps times (and the e4m3 correction term in "
                                 "its sweeps)"}}
    line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
    print(json.dumps(line))
    return 0


def threed_workload(args):
    """The 3-D operator: 34 x 34 x 34 nodes (32^3 = 32768 unknowns), lognormal
    node eps, B = 1024 Gaussian charges, refined BF16 with the sweep count
    calibrated to Eq. 6 error <= 0.5e-6 against the FP64 GPU apply; one step =
    one refined apply of the batch, inputs resident in HBM."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_00001_gb300.binding import Solver3D
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    N, B = (args.nodes if args.nodes != NODES else 34), args.batch
    h = 1.0 / (N - 1)
    rng = np.random.default_rng(3)
    eps = np.exp(0.5 * rng.standard_normal((N, N, N)))
    # B Gaussian charges at random centres, width 0.05
    z, y, x = np.meshgrid(*(h * np.arange(1, N - 1),) * 3, indexing="ij")
    ctr = rng.uniform(0.2, 0.8, (B, 3))
    amp = rng.standard_normal(B)
    rho = np.stack([a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * 0.05 ** 2))
                    for a, c in zip(amp, ctr)]).reshape(B, -1)
    s64 = Solver3D(N, N, N, h, eps, "fp64")
    b = s64.rhs_from_charge(torch.from_numpy(rho).cuda())
    cols = list(range(0, B, max(B // 16, 1)))[:16]
    ref = s64.apply(b[cols].contiguous())
    setup64 = s64.info().setup_ms
    s64.close()
    torch.cuda.empty_cache()
    # 3-D: FP16 alone reaches the target in one sweep (34^3 nodes: 348k solves/s;
    # with the correction term 282k, BF16 215k in two sweeps), so FP16 is the default
    prec = args.precision if args.precision in ("bf16", "bf16_fp8", "fp16", "fp16_fp8") else "fp16"
    s = Solver3D(N, N, N, h, eps, prec)
    tune = dict(kv.split("=", 1) for kv in args.tune)
    if tune:
        s.set_tuning(**{kk: int(v) for kk, v in tune.items()})
    s.reserve(B)
    u = torch.empty_like(b)
    errs = {}
    k = args.sweeps
    if k < 0:
        for kk in range(16):
            s.apply(b, u, sweeps=kk)
            e = float(((u[cols] - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max())
            errs[str(kk)] = e
            if e <= TARGET_ERR:
                k = kk
                break
        k = 15 if k < 0 else k
    for _ in range(max(args.warmup, 1)):
        s.apply(b, u, sweeps=k)
    torch.cuda.synchronize()
    with s.profile() as prof:
        ms = _evt_time(lambda: s.apply(b, u, sweeps=k), args.steps)
    err = float(((u[cols] - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max())
    n = s.n
    la, ams = prof["apply"]
    pk, pk_kind = peaks()
    achieved = 2.0 * n * n * B / (ams / la * 1e-3) / 1e12 if la else 0.0
    line = {"metric": "RHS solves/s, 3-D 32^3 interior (34^3 nodes), B=1024, refined FP16/BF16/FP8 @1e-6",
            "value": B / (ms * 1e-3), "unit": "RHS solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"{N}^3 nodes, lognormal eps, {B} Gaussian charges",
                       "unknowns": n, "sweeps": k, "setup_ms_fp64": setup64,
                       "setup_ms_bf16": s.info().setup_ms},
            "accuracy": {"max_rel_err_eq6_vs_fp64": err, "target": 1e-6, "err_by_sweeps": errs},
            "kernel_ms_per_step": {c: prof[c][1] / (args.steps + 1) for c in prof},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
                         "frac_of_sustained": achieved / pk["bf16_tflops_sustained"],
                         "traffic": None, "peak_source": f"{pk_kind} bf16_tflops (burst)"}}
    print(json.dumps(line))
    return 0


def formats_workload(args):
    """Table 1 on the GPU and its extension to the binary stored formats.

    (a) The Eq. (4)/(5) problem on n x n nodes, n in {5, 11, 21, 41, 81}: the
    FP64 inverse formed on the GPU, rounded to k decimals on the GPU, one FP64
    apply, Eq. (6) error; beside the printed value.  (b) For FP32, BF16, BF16 with
    the e4m3 correction term, FP8 and FP8 hi+lo stores, Fourier-field eps, 16
    right-hand sides: Eq. (6) error
    against the FP64 GPU apply after k refinement sweeps, the contraction per
    sweep and the sweeps needed for 1e-6, on grids from 21^2 to 200^2 nodes."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_00001_gb300 import workloads as W
    from paper_1602_00001_gb300.binding import Solver
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    golden = os.path.join(ROOT, "tests", "golden", "table1.txt")
    printed = {}
    for ln in open(golden):
        if ln.startswith("#") or not ln.strip():
            continue
        parts = ln.split()
        for n, v in zip([5, 11, 21, 41, 81], parts[1:]):
            printed[(n, parts[0])] = v
    table, match = {}, 0
    t0 = time.perf_counter()
    for n in [5, 11, 21, 41, 81]:
        h = 1.0 / (n - 1)
        x = h * np.arange(n)
        X, Y = np.meshgrid(x, x)
        f = W.example_source(X, Y)[1:-1, 1:-1].reshape(1, -1)
        ua = W.example_exact(X, Y)
        for k in ["1", "2", "3", "5", "none"]:
            s = Solver(n, n, h, np.ones((n, n)), "fp64")
            b = s.rhs_from_charge(f)
            if k != "none":
                s.round_inverse_decimal(int(k))
            u = np.zeros((n, n))
            u[1:-1, 1:-1] = s.apply(b).cpu().numpy().reshape(n - 2, n - 2)
            err = float(np.max(np.abs(ua - u)) / np.max(np.abs(ua)))
            p = printed[(n, k)]
            ok = abs(err - float(p)) <= 0.5 * 10.0 ** (-len(p.split(".")[1])) + 1e-12
            match += int(ok)
            table[f"n={n},digits={k}"] = {"gpu": err, "printed": float(p), "match": ok}
            s.close()
    t_table = time.perf_counter() - t0
    study = {}
    B = 16
    for N in [21, 41, 81, 161, 200]:
        h = 1.0 / (N - 1)
        eps = W.eps_fourier(N, N, h, seed=1)
        rho = W.moving_charges(N, N, h, seed=5, steps=B)
        s64 = Solver(N, N, h, eps, "fp64")
        b = s64.rhs_from_charge(torch.from_numpy(rho).cuda())
        ref = s64.apply(b)
        s64.close()
        row = {}
        for prec in ["fp32", "bf16", "bf16_fp8", "bf16_fp8_every_sweep", "fp16", "fp16_fp8",
                     "fp8", "fp8x2"]:
            # bf16_fp8: the correction term in the first sweep (its default);
            # bf16_fp8_every_sweep: in the first apply and every sweep;
            # fp16_fp8: in the first apply (its default)
            s = Solver(N, N, h, eps, "bf16_fp8" if prec.startswith("bf16_fp8") else prec)
            if prec == "bf16_fp8_every_sweep":
                s.set_tuning(corr_mask=(1 << 30) - 1)
            errs = []
            for k in range(0, 9):
                u = s.apply(b, sweeps=k)
                errs.append(float(((u - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max()))
                if errs[-1] < 1e-13:
                    break
            # ratios of consecutive sweeps while the error is well above the FP64
            # floor (~1e-13): below ~1e-10 the ratio measures rounding, not contraction
            ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1) if errs[i + 1] > 1e-10]
            need = next((k for k, e in enumerate(errs) if e <= 1e-6), None)
            row[prec] = {"err_by_sweeps": errs, "store_bytes": s.info().store_bytes,
                         "contraction": float(np.median(ratios)) if ratios else None,
                         "sweeps_for_1e-6": need}
            s.close()
        study[f"{N}x{N}"] = row
    line = {"metric": "Table 1 cells reproduced on the GPU (of 25)", "value": match,
            "unit": "cells", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": t_table * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "Table 1 (Eq. 4/5, n = 5..81, digits 1, 2, 3, 5, none) and "
                                   "stored-format study (Fourier eps, 16 moving charges, "
                                   "21^2..200^2 nodes)"},
            "table1": table, "formats": study}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default=None,
                    choices=["auto", "bf16", "bf16_fp8", "fp16", "fp16_fp8", "fp8x2", "fp32"],
                    help="stored format (default: auto -- chosen by the library from the measured "
                         "contraction -- for the 2-D apply; fp16_fp8 for the adjoint, fp16 in 3-D)")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--sweeps", type=int, default=-1, help="fixed sweep count (-1: calibrate)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--nodes", type=int, default=NODES, help="grid nodes per side (profiling runs)")
    ap.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                    help="launch-shape knob of the refined solver (pide_set_tuning), repeatable")
    ap.add_argument("--workload", default="apply",
                    choices=["apply", "batched", "adjoint", "formats", "3d"],
                    help="apply: the headline (default); batched / adjoint / formats: other rows")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_workload(args)
    if args.workload == "adjoint":
        return adjoint_workload(args)
    if args.workload == "formats":
        return formats_workload(args)
    if args.workload == "3d":
        return threed_workload(args)
    if args.precision is None:
        args.precision = PRECISION

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_00001_gb300 import workloads as W
    from paper_1602_00001_gb300.binding import Solver

    B = args.batch
    NN = args.nodes
    h = 1.0 / (NN - 1)
    eps = W.eps_fourier(NN, NN, h, seed=5)
    rho_np = W.moving_charges(NN, NN, h, seed=5 + rank, steps=B)
    stream = torch.cuda.current_stream()

    # ---- the plain FP64 GPU apply: reference solution for sampled columns and
    #      the comparator rate (FP64 is compute bound at any B on this part)
    s64 = Solver(NN, NN, h, eps, "fp64")
    rho = torch.from_numpy(rho_np).cuda()
    b = s64.rhs_from_charge(rho)
    sample_cols = list(range(0, B, max(B // 16, 1)))[:16]
    b_s = b[sample_cols].contiguous()
    u64_s = s64.apply(b_s)
    torch.cuda.synchronize()

    def timed(fn, reps):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        z.record()
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    fp64_b1_ms = timed(lambda: s64.apply(b[:1].contiguous()), 5)
    b64c = b[:64].contiguous()
    fp64_b64_ms = timed(lambda: s64.apply(b64c), 3)
    # the whole batch through the FP64 apply (B = 1024: ~3 s per apply on the FP64 pipe)
    fp64_bB_ms = None
    if NN == NODES and B == BATCH:
        u64_all = torch.empty_like(b)
        fp64_bB_ms = timed(lambda: s64.apply(b, u64_all), 3)
        del u64_all
    s64.close()
    del s64
    torch.cuda.empty_cache()
    # FP64 peak of this GPU: cuBLAS DGEMM through torch (4096^3, best of 5)
    Ad = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    fp64_gemm_ms = min(timed(lambda: torch.matmul(Ad, Ad), 1) for _ in range(5))
    fp64_peak_tf = 2.0 * 4096 ** 3 / (fp64_gemm_ms * 1e-3) / 1e12
    del Ad
    # e4m3 peak of this GPU: cuBLASLt FP8 GEMM through torch._scaled_mm (8192^3, best of
    # 5), the denominator of the correction GEMM when it runs; else the nominal ratio
    fp8_peak_tf = None
    try:
        A8 = torch.randn(8192, 8192, device="cuda").to(torch.float8_e4m3fn)
        B8 = torch.randn(8192, 8192, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        fp8_ms = min(timed(lambda: torch._scaled_mm(A8, B8, one, one, out_dtype=torch.bfloat16), 2)
                     for _ in range(5))
        fp8_peak_tf = 2.0 * 8192 ** 3 / (fp8_ms * 1e-3) / 1e12
        del A8, B8
    except Exception:
        fp8_peak_tf = None
    torch.cuda.empty_cache()

    # ---- the refined low-precision solver (the store chosen by the library unless forced)
    s = Solver(NN, NN, h, eps, args.precision)
    auto_rep = s.auto_report() if args.precision == "auto" else None
    args.precision = s.precision
    tune = dict(kv.split("=", 1) for kv in args.tune)
    if tune:
        s.set_tuning(**{k: int(v) for k, v in tune.items()})
    s.reserve(B)
    n = s.n
    u = torch.empty((B, n), dtype=torch.float64, device="cuda")

    def err_of(uu):
        d = (uu[sample_cols] - u64_s).abs().amax(dim=1) / u64_s.abs().amax(dim=1)
        return float(d.max())

    calib = {}
    if args.sweeps >= 0:
        k = args.sweeps
        s.apply(b, u, sweeps=k)
        err = err_of(u)
    else:
        k, err = None, None
        for kk in range(0, 16):
            s.apply(b, u, sweeps=kk)
            e = err_of(u)
            calib[kk] = e
            if e <= TARGET_ERR:
                k, err = kk, e
                break
        if k is None:
            k, err = 15, e
    # B = 1 on the same grid (GEMV path), calibrated the same way
    b1 = b[:1].contiguous()
    u1 = torch.empty((1, n), dtype=torch.float64, device="cuda")
    k1 = 15
    for kk in range(0, 16):
        s.apply(b1, u1, sweeps=kk)
        e1 = float(((u1[0] - u64_s[0]).abs().max() / u64_s[0].abs().max()))
        if e1 <= TARGET_ERR:
            k1 = kk
            break

    # the refinement's measured contraction on this batch (pide_info), outside the timed region
    _, info_k = s.apply(b, u, sweeps=k, want_info=True)

    # ---- timed region: K steps of the whole refined batch
    for _ in range(args.warmup):
        s.apply(b, u, sweeps=k)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        with s.profile() as prof:
            torch.cuda.synchronize()
            e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            # an NVTX range around the timed steps lets a profiler select them
            torch.cuda.nvtx.range_push("timed_steps")
            for _ in range(args.steps):
                s.apply(b, u, sweeps=k)
            torch.cuda.nvtx.range_pop()
            e1_.record(stream)
            torch.cuda.synchronize()
        ms_total = e0.elapsed_time(e1_)
    if dist:
        ms_total = reduce_max(ms_total, dist)
        dist.barrier()
    ms_step = ms_total / args.steps
    value = whole_job_rate(world, B, args.steps, ms_total)
    err_final = err_of(u)

    pk, pk_kind = peaks()
    # B = 1 rate, and the HBM roofline of its apply kernel (live CUDA events)
    b1_ms = timed(lambda: s.apply(b1, u1, sweeps=k1), 10)
    with s.profile() as prof1:
        for _ in range(5):
            s.apply(b1, u1, sweeps=k1)
    b1_apply_launches, b1_apply_ms = prof1["apply"]
    hi = s.info()
    hi64_bytes = 8 * n * hi.ld
    sym_b1 = args.precision in ("bf16", "bf16_fp8", "fp16", "fp16_fp8") and s.get_tuning()["symv"]
    b1_bytes = hi.store_bytes if not sym_b1 else \
        2 * 2 * (((n + 127) // 128) * (((n + 127) // 128) + 1) // 2) * 128 * 128
    b1_gbs = b1_bytes * b1_apply_launches / (b1_apply_ms * 1e-3) / 1e9

    # ---- the other batch sizes of the metric's definition (B = 64, 4096), same sweeps:
    #      B = 64 columns of the batch; B = 4096 the batch four times over
    batch_sweep = {}
    if NN == NODES and B == BATCH:
        for Bx in (64, 4096):
            bx = b[:Bx].contiguous() if Bx <= B else b.repeat((Bx + B - 1) // B, 1)[:Bx].contiguous()
            ux = torch.empty_like(bx)
            s.reserve(Bx)
            msx = timed(lambda: s.apply(bx, ux, sweeps=k), 5)
            ex = float(((ux[:min(Bx, len(sample_cols))] - u[:min(Bx, len(sample_cols))]).abs()
                        .amax(dim=1) / u[:min(Bx, len(sample_cols))].abs().amax(dim=1)).max())
            batch_sweep[str(Bx)] = {"value": world * Bx / (msx * 1e-3), "unit": UNIT,
                                    "ms_per_step": msx, "sweeps": k,
                                    "max_rel_diff_vs_b1024_columns": ex}
            del bx, ux
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI from pinned host memory, copies inside the timed
    #      region: pide_solve_stream over E_BATCHES steps of B columns (each step's input
    #      copied in and its solution copied out, overlapping the neighbouring steps' solves)
    # 8 steps of B per call: a time sequence of 8B right-hand sides, whose first and
    # last half-chunk copies are the only ones not hidden under a solve
    E_BATCHES = 8
    b_host = b.cpu().pin_memory()
    in_host = torch.empty((E_BATCHES * B, n), dtype=torch.float64).pin_memory()
    for e in range(E_BATCHES):
        in_host[e * B:(e + 1) * B].copy_(b_host)
    u_host = torch.empty((E_BATCHES * B, n), dtype=torch.float64).pin_memory()
    s.solve_stream(in_host, u_host, chunk=B, sweeps=k)          # allocates the device slots
    torch.cuda.synchronize()
    # seven timed calls; the median call is reported, every call's rate beside it
    # (host-side copy rates vary between calls on a shared machine)
    call_rates = []
    for _ in range(7):
        t0 = time.perf_counter()
        s.solve_stream(in_host, u_host, chunk=B, sweeps=k)
        dt = reduce_max((time.perf_counter() - t0) / E_BATCHES, dist)
        call_rates.append(world * B / dt)
    e2e_value = sorted(call_rates)[len(call_rates) // 2]
    ud = u[sample_cols].cpu()
    e2e_err = float(((u_host[(E_BATCHES - 1) * B:][sample_cols] - ud).abs().amax(dim=1)
                     / ud.abs().amax(dim=1)).max())
    # one batch per call through pide_apply_host (no overlap across calls), for context
    u1_host = torch.empty_like(b_host).pin_memory()
    s.apply_host(b_host, u1_host, sweeps=k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        s.apply_host(b_host, u1_host, sweeps=k)
    ah_value = world * B / reduce_max((time.perf_counter() - t0) / 3, dist)
    del in_host, u_host

    # ---- roofline of the dominant kernel (the apply GEMM), from live CUDA events
    apply_launches, apply_ms = prof["apply"]
    gemm_ms = apply_ms / max(apply_launches, 1)
    # every timed step applies the stored inverse (1 + k) times to all B columns
    # (as one launch or as two column-group launches when the residual overlaps);
    # FP8X2 contracts the hi and the lo term: twice the flops, on the FP8 pipe
    terms = 2 if args.precision == "fp8x2" else 1
    flops_total = 2.0 * n * n * B * (1 + k) * args.steps * terms
    achieved = flops_total / (apply_ms * 1e-3) / 1e12
    # The GEMM launches (~1.9 ms each) are timed inside a 5 ms step and a timed region
    # of a fraction of a second: the burst figure is the denominator; the fraction of
    # the seconds-long sustained figure (power-capped) is reported beside it.
    if args.precision == "fp8x2":
        ratio = 2.0                                        # nominal FP8:BF16 dense ratio 4.5:2.25
        peak_src = f"{pk_kind} bf16_tflops (burst) x 2 (nominal FP8/BF16 ratio)"
    else:
        ratio = 1.0
        peak_src = f"{pk_kind} bf16_tflops (burst)"
        if args.precision.startswith("fp16"):
            peak_src += " (FP16 and BF16 share the dense tensor rate: nominal ratio 1)"
    peak_tf = pk["bf16_tflops"] * ratio
    sustained_tf = pk["bf16_tflops_sustained"] * ratio
    traffic = None
    tn = s.get_tuning()
    traffic_valid = (gemm_source_sha1() == GEMM_TRAFFIC["sha1"]
                     and args.precision == GEMM_TRAFFIC["precision"] and k == GEMM_TRAFFIC["sweeps"]
                     and B == GEMM_TRAFFIC["batch"] and NN == GEMM_TRAFFIC["nodes"]
                     and tn["corr_mask"] == GEMM_TRAFFIC["corr_mask"] and tn["gemm_2cta"] == 1
                     and tn["gemm_a_hint"] == GEMM_TRAFFIC["a_hint"] and tn["gemm_u_hint"] == 1)
    if traffic_valid:
        traffic = GEMM_TRAFFIC["bytes"]
    launches = sum(prof[c][0] for c in prof)
    # PIDE_BF16_FP8: the correction term's e4m3 GEMM (profile class "other") on the FP8 pipe
    corr_line = None
    if args.precision.endswith("_fp8") and prof["other"][0] > 0:
        c_launches, c_ms = prof["other"]
        c_tf = 2.0 * n * n * B * c_launches / (c_ms * 1e-3) / 1e12
        c_peak = fp8_peak_tf if fp8_peak_tf else pk["bf16_tflops"] * 2.0
        corr_line = {"kernel": "gemm_tc2_kernel (tcgen05 cta_group::2 e4m3 correction term)",
                     "launches": c_launches, "avg_launch_ms": c_ms / c_launches,
                     "achieved": c_tf, "peak": c_peak, "unit": "TFLOP/s", "frac": c_tf / c_peak,
                     "frac_of_sustained": c_tf / (pk["bf16_tflops_sustained"] * 2.0),
                     "peak_source": ("cuBLASLt e4m3 GEMM through torch._scaled_mm, 8192^3, "
                                     "best of 5, measured in this run") if fp8_peak_tf else
                                    f"{pk_kind} bf16_tflops (burst) x 2 (nominal FP8/BF16 ratio)",
                     "corr_mask": s.get_tuning()["corr_mask"],
                     "traffic": GEMM_TRAFFIC["corr_bytes"] if traffic_valid else None}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": WORKLOAD if NN == NODES else f"{NN - 2}^2 interior, B={B}",
                   "global_batch": B * world, "per_gpu_batch": B,
                   "grid": f"{NN}x{NN}", "unknowns": n, "precision": args.precision,
                   "sweeps": k, "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({hi.store_bytes / 1e9:.2f} GB stored inverse "
                         f"({args.precision}) streamed per apply)"},
        "accuracy": {"max_rel_err_eq6_vs_fp64": err_final, "target": 1e-6,
                     "sampled_columns": len(sample_cols),
                     "err_by_sweeps": {str(kk): v for kk, v in calib.items()}},
        "b1": {"value": 1.0 / (b1_ms * 1e-3), "unit": UNIT, "sweeps": k1, "ms": b1_ms,
               "path": "symmetric S^-1, BF16 hi+lo packed lower tiles" if sym_b1 else "GEMV over the stored L^-1",
               "roofline": {"bound": "hbm", "achieved": b1_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": b1_gbs / pk["hbm_gbs"], "bytes_per_apply": b1_bytes,
                            "avg_apply_ms": b1_apply_ms / max(b1_apply_launches, 1)}},
        "fp64_gpu": {"b1_solves_per_s": 1.0 / (fp64_b1_ms * 1e-3),
                     "b64_solves_per_s": 64.0 / (fp64_b64_ms * 1e-3),
                     "b1024_solves_per_s": (B / (fp64_bB_ms * 1e-3)) if fp64_bB_ms else None,
                     "b1024_ms": fp64_bB_ms, "b1024_repeats": 3 if fp64_bB_ms else 0,
                     "speedup_b1024_vs_fp64": (value / world / (B / (fp64_bB_ms * 1e-3)))
                                              if fp64_bB_ms else None,
                     "speedup_b1_vs_fp64": fp64_b1_ms / b1_ms,
                     "fp64_peak_tflops": fp64_peak_tf,
                     "fp64_peak_source": "cuBLAS DGEMM through torch.matmul, 4096^3, best of 5",
                     "b1_fp64_tflops": 2.0 * n * n / (fp64_b1_ms * 1e-3) / 1e12,
                     "b1024_fp64_tflops": (2.0 * n * n * B / (fp64_bB_ms * 1e-3) / 1e12)
                                          if fp64_bB_ms else None,
                     "b1_hbm_gbs": hi64_bytes / (fp64_b1_ms * 1e-3) / 1e9,
                     "bound": "FP64 pipe: n^2 FP64 multiply-adds per column at B = 1 "
                              "(the 12.3 GB inverse would stream in 1.8 ms at the HBM peak)"},
        "peaks_in_run": {"fp64_tflops": fp64_peak_tf, "fp8_e4m3_tflops": fp8_peak_tf,
                         "how": "cuBLAS DGEMM 4096^3 and cuBLASLt e4m3 GEMM 8192^3 through "
                                "torch, best of 5, before the timed region"},
        "contraction": {"measured": info_k.contraction, "sweeps": info_k.sweeps,
                        "rel_residual": info_k.rel_residual, "apply_ms": info_k.ms,
                        "source": "pide_info of one refined apply of the batch"},
        "store": {"precision": args.precision,
                  "chosen_by": "pide_setup_auto (measured contraction)" if auto_rep else "--precision",
                  "auto": auto_rep},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf, "frac_of_sustained": achieved / sustained_tf,
                     "traffic": traffic,
                     "traffic_source": GEMM_TRAFFIC["source"] if traffic else None,
                     "kernel": (f"gemm_tc2_kernel (tcgen05 cta_group::2 {args.precision}, M=256 N=256 per SM pair)"
                                if s.get_tuning()["gemm_2cta"] and B > 128 else
                                f"gemm_tc_kernel (tcgen05 {args.precision}, M=128 N=256)"),
                     "peak_source": peak_src,
                     "avg_launch_ms": gemm_ms, "launches": apply_launches,
                     "algorithmic_flops_per_launch": flops_total / max(apply_launches, 1)},
        "kernel_ms_per_step": {c: prof[c][1] / args.steps for c in prof},
        "correction_gemm": corr_line,
        "other_batch_sizes": batch_sweep,
        "overlap": bool(s.get_tuning()["overlap"]),
        "tuning": s.get_tuning(),
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * n * 8,
                "d2h_bytes_per_step": B * n * 8,
                "api": f"pide_solve_stream, {E_BATCHES} steps of B={B} per call, pinned host buffers",
                "calls": call_rates, "reported": "median of the calls",
                "max_rel_diff_vs_device_apply": e2e_err,
                "apply_host_one_batch_per_call": ah_value},
    }
    # ---- the oracle on the host cores (rank 0, N = 1 only), bounded sample
    if rank == 0 and world == 1 and not args.no_cpu and NN == NODES and B == BATCH:
        from oracle import pide_oracle as O
        cores = max(1, min(os.cpu_count() or 1, BATCH // 4))
        cpu_line, u_or = cpu_baseline_leg(NN, 5, cores, cols=4)
        ur = u[:4].cpu().numpy()
        line["accuracy"]["max_rel_err_eq6_vs_oracle_4col"] = O.rel_error_eq6(ur, u_or)
        line["cpu_baseline"] = cpu_line
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
