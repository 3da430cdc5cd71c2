"""Autotuner for the apply kernels' launch shapes.

For a (grid size bucket, column-count bucket, precision) key it times every
candidate setting of the library's tuning knobs (pide_set_tuning) with CUDA
events on the launching stream and keeps the fastest.  Results live in a JSON
cache keyed by GPU name (path: $PIDE_TUNE_CACHE, default
~/.cache/pide_tune.json) so later processes reuse them without timing.

Knobs: for B > 128 the SM-pair GEMM (256 x 256 tiles) against the single-SM
one (tile width 128/256), the stream-K tail (on/off) and the L2 policy of the
streamed inverse; GEMV block size (256..1024) and loads in flight (4/8) for
B = 1; the largest B sent to the GEMV instead of the tensor-core GEMM (1..8).
The knobs change only the launch shape, never the arithmetic beyond FP32
summation order.
"""
from __future__ import annotations

import itertools
import json
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pide_tune.json")


def cache_path() -> str:
    return os.environ.get("PIDE_TUNE_CACHE", DEFAULT_CACHE)


def bucket_n(n: int) -> str:
    """Power-of-two bucket of the unknown count."""
    b = 1
    while b < n:
        b <<= 1
    return f"n<={b}"


def bucket_b(B: int) -> str:
    if B <= 1:
        return "B=1"
    if B <= 8:
        return "B<=8"
    if B <= 128:
        return "B<=128"
    if B <= 1024:
        return "B<=1024"
    return "B>1024"


def key_for(n: int, B: int, precision: str) -> str:
    return f"{precision}|{bucket_n(n)}|{bucket_b(B)}"


def candidates(B: int):
    """Candidate knob settings for a column count (dicts of solver knobs)."""
    if B <= 1:
        for th, un in itertools.product([256, 512, 1024], [4, 8]):
            yield {"gemv_max_b": 1, "gemv_threads": th, "gemv_unroll": un}
    elif B <= 8:
        yield {"gemv_max_b": 1}
        for th in (512, 1024):
            yield {"gemv_max_b": 8, "gemv_threads": th, "gemv_unroll": 8}
    elif B <= 128:
        for sk in (0, 1):
            yield {"gemv_max_b": 1, "gemm_streamk": sk}
    else:
        # SM pairs: whole tiles, the K-split last round weighed against its
        # reduction, or split whenever the round gets shorter; the inverse's
        # loads with an L2 evict-normal or evict-last hint (evict-first
        # doubled the pair kernel's DRAM reads)
        for sk, hint in itertools.product([0, 1, 2], [1, 2]):
            yield {"gemv_max_b": 1, "gemm_2cta": 1, "gemm_bn": 256, "gemm_streamk": sk,
                   "gemm_a_hint": hint}
        for bn, sk in itertools.product([128, 256], [0, 1]):
            yield {"gemv_max_b": 1, "gemm_2cta": 0, "gemm_bn": bn, "gemm_streamk": sk,
                   "gemm_a_hint": 0}


class TuneCache:
    """JSON file: {gpu_name: {key: {"knobs": {...}, "ms": float}}}."""

    def __init__(self, path: str | None = None):
        self.path = path or cache_path()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, gpu: str, key: str):
        return self.data.get(gpu, {}).get(key)

    def put(self, gpu: str, key: str, knobs: dict, ms: float):
        self.data.setdefault(gpu, {})[key] = {"knobs": dict(knobs), "ms": float(ms)}

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def search(cands, timer):
    """Return (best_knobs, best_ms, all) for a timer(knobs) -> ms callable."""
    results = []
    for k in cands:
        results.append((timer(k), k))
    results.sort(key=lambda t: t[0])
    return results[0][1], results[0][0], results


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def event_timer(solver, b, sweeps: int = 0, reps: int = 3):
    """Timer for real runs: CUDA events around `reps` applies on the current stream."""
    import torch

    def t(knobs):
        solver.set_tuning(**knobs)
        solver.apply(b, sweeps=sweeps)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            solver.apply(b, sweeps=sweeps)
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    return t


def tune(solver, b, cache: TuneCache | None = None, gpu: str | None = None, timer=None,
         save: bool = True):
    """Tune the knobs for this solver and right-hand-side block; apply the
    winner to the solver and record it in the cache.  Returns (knobs, ms)."""
    B = b.reshape(-1, solver.n).shape[0]
    cache = cache or TuneCache()
    gpu = gpu or _gpu_name()
    timer = timer or event_timer(solver, b)
    best, ms, _ = search(candidates(B), timer)
    cache.put(gpu, key_for(solver.n, B, solver.precision), best, ms)
    if save:
        cache.save()
    solver.set_tuning(**best)
    return best, ms


def apply_cached(solver, B: int, cache: TuneCache | None = None, gpu: str | None = None) -> bool:
    """Set the cached knobs for (solver, B) if the cache has them."""
    cache = cache or TuneCache()
    ent = cache.get(gpu or _gpu_name(), key_for(solver.n, B, solver.precision))
    if not ent:
        return False
    solver.set_tuning(**ent["knobs"])
    return True


# ---------------------------------------------------------------- batched plans
# The knobs a batched plan reads from each problem's handle when it is created:
# for BF16 problems and FP32 problems on the TF32 tensor cores the grouped
# launch's column-tile width (32, 64, 128); for FP32 problems also the SIMT
# tiles (FP32 products, width 16, 32, 64) instead of the tensor cores.


def bucket_b_batch(B: int) -> str:
    """Column-count bucket of the batched-plan knobs: one per column-tile width
    that covers B in one tile (a problem with 33..64 columns needs two 32-wide
    tiles, each streaming the inverse again), so a finer split than bucket_b."""
    for top in (8, 16, 32, 64, 128):
        if B <= top:
            return f"B<={top}"
    return "B>128"


def batch_key_for(n: int, B: int, precision: str) -> str:
    return f"batch|{precision}|{bucket_n(n)}|{bucket_b_batch(B)}"


def batch_candidates(precision: str, B: int):
    for bn in (32, 64, 128):
        if bn >= 2 * max(B, 16) and bn > 32:
            continue               # wider than twice the columns: idle tensor columns
        yield {"batch_tc": 1, "batch_bn": bn}
    if precision == "fp32":
        for tn in (16, 32, 64):
            yield {"batch_tc": 0, "batch_tn": tn}


def batch_plan_timer(solver, b, u, sweeps: int, reps: int = 5):
    """Timer for one problem alone in a plan: CUDA events around `reps` runs
    (a new plan per candidate, since plans read the knobs when created)."""
    import torch
    from .binding import BatchPlan

    def t(knobs):
        solver.set_tuning(**knobs)
        plan = BatchPlan([solver], [b], [u])
        plan.run(sweeps=sweeps, use_graph=False)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            plan.run(sweeps=sweeps, use_graph=False)
        e.record()
        torch.cuda.synchronize()
        plan.close()
        return s.elapsed_time(e) / reps

    return t


def tune_batch(solver, b, u, sweeps: int = 2, cache: TuneCache | None = None,
               gpu: str | None = None, timer=None, save: bool = True):
    """Tune the batched-plan knobs of one problem (its solver, right-hand sides
    b and output u, [B][n] device tensors); the winner is set on the solver and
    cached under the (precision, n bucket, B bucket) key.  Returns (knobs, ms)."""
    B = b.reshape(-1, solver.n).shape[0]
    cache = cache or TuneCache()
    gpu = gpu or _gpu_name()
    timer = timer or batch_plan_timer(solver, b, u, sweeps)
    best, ms, _ = search(batch_candidates(solver.precision, B), timer)
    cache.put(gpu, batch_key_for(solver.n, B, solver.precision), best, ms)
    if save:
        cache.save()
    solver.set_tuning(**best)
    return best, ms


def apply_cached_batch(solver, B: int, cache: TuneCache | None = None,
                       gpu: str | None = None) -> bool:
    """Set the cached batched-plan knobs for (solver, B) if the cache has them."""
    cache = cache or TuneCache()
    ent = cache.get(gpu or _gpu_name(), batch_key_for(solver.n, B, solver.precision))
    if not ent:
        return False
    solver.set_tuning(**ent["knobs"])
    return True
