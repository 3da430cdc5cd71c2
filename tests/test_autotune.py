"""Autotuner: candidate sets, search, the JSON cache (CPU, fake timer), and
one real tuning pass on the GPU."""
import json

import numpy as np
import pytest

from paper_1602_00001_gb300 import autotune as T


class FakeSolver:
    n = 39204
    precision = "bf16"

    def __init__(self):
        self.knobs = {}

    def set_tuning(self, **kv):
        self.knobs.update(kv)


class FakeB:
    def __init__(self, B):
        self.shape = (B, 39204)

    def reshape(self, *a):
        return self


def test_keys_and_buckets():
    assert T.bucket_n(39204) == "n<=65536"
    assert T.bucket_b(1) == "B=1" and T.bucket_b(1024) == "B<=1024" and T.bucket_b(4096) == "B>1024"
    assert T.key_for(2304, 64, "fp8x2") == "fp8x2|n<=4096|B<=128"


@pytest.mark.parametrize("B", [1, 5, 64, 1024])
def test_candidates_are_valid_knobs(B):
    c = list(T.candidates(B))
    assert c
    for k in c:
        assert set(k) <= {"gemv_max_b", "gemv_threads", "gemv_unroll", "gemm_bn", "gemm_streamk",
                          "gemm_2cta", "gemm_a_hint"}


def test_tune_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    cache = T.TuneCache(path)
    s = FakeSolver()

    def timer(knobs):  # pretend BN=256 with stream-K is fastest
        return 1.0 + (knobs.get("gemm_bn") != 256) + 0.5 * (knobs.get("gemm_streamk") != 1)

    best, ms = T.tune(s, FakeB(1024), cache=cache, gpu="GB300", timer=timer)
    assert best["gemm_bn"] == 256 and best["gemm_streamk"] == 1 and ms == 1.0
    assert s.knobs["gemm_bn"] == 256
    data = json.load(open(path))
    assert data["GB300"]["bf16|n<=65536|B<=1024"]["ms"] == 1.0
    s2 = FakeSolver()
    assert T.apply_cached(s2, 1024, cache=T.TuneCache(path), gpu="GB300")
    assert s2.knobs == best
    assert not T.apply_cached(s2, 1, cache=T.TuneCache(path), gpu="GB300")


def test_corrupt_cache_is_ignored(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert T.TuneCache(str(p)).data == {}


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    import torch
    from paper_1602_00001_gb300 import build, workloads as W
    from paper_1602_00001_gb300.binding import Solver
    build.build()
    n = 60
    h = 1.0 / (n - 1)
    s = Solver(n, n, h, W.eps_lognormal(n, n, 2), "bf16")
    b = torch.from_numpy(W.random_interior(n, n, 1, batch=300)).cuda()
    u_ref = s.apply(b, sweeps=3)
    best, ms = T.tune(s, b, cache=T.TuneCache(str(tmp_path / "t.json")))
    assert ms > 0 and s.get_tuning()["gemm_bn"] == best["gemm_bn"]
    u = s.apply(b, sweeps=3)
    assert float((u - u_ref).abs().max()) <= 1e-6 * float(u_ref.abs().max())


@pytest.mark.parametrize("prec,B", [("fp32", 1), ("fp32", 64), ("bf16", 9)])
def test_batch_candidates_are_valid_knobs(prec, B):
    c = list(T.batch_candidates(prec, B))
    assert c and all(set(k) <= {"batch_tc", "batch_bn", "batch_tn"} for k in c)
    assert all(k["batch_bn"] in (32, 64, 128) for k in c if k.get("batch_tc") == 1)
    assert any(k.get("batch_tc") == 0 for k in c) == (prec == "fp32")


def test_tune_batch_caches_and_applies(tmp_path):
    path = str(tmp_path / "tune.json")
    s = FakeSolver()
    s.precision = "fp32"

    def timer(knobs):  # pretend the 128-wide tensor-core tiles are fastest
        return 1.0 if knobs == {"batch_tc": 1, "batch_bn": 128} else 2.0

    best, ms = T.tune_batch(s, FakeB(100), None, cache=T.TuneCache(path), gpu="GB300", timer=timer)
    assert best == {"batch_tc": 1, "batch_bn": 128} and ms == 1.0
    assert json.load(open(path))["GB300"]["batch|fp32|n<=65536|B<=128"]["knobs"] == best
    assert T.batch_key_for(1000, 40, "bf16") == "batch|bf16|n<=1024|B<=64"
    assert T.batch_key_for(1000, 32, "bf16") == "batch|bf16|n<=1024|B<=32"
    s2 = FakeSolver()
    s2.precision = "fp32"
    assert T.apply_cached_batch(s2, 100, cache=T.TuneCache(path), gpu="GB300")
    assert s2.knobs == best


@pytest.mark.gpu
def test_tuned_cache_entry_changes_the_plan_shape(tmp_path):
    """A batched-plan entry in the tuner's cache reaches pide_batch_create: the
    plan built with the cache launches the cached column-tile width."""
    import torch
    from paper_1602_00001_gb300 import build, workloads as W
    from paper_1602_00001_gb300.binding import BatchPlan, Solver
    build.build()
    n = 40
    s = Solver(n, n, 1.0 / (n - 1), W.eps_lognormal(n, n, 3), "fp32")
    b = torch.from_numpy(W.random_interior(n, n, 2, batch=20)).cuda()
    u = torch.empty_like(b)
    plain = BatchPlan([s], [b], [u])
    assert plain.info()["tc_items_bn"] == {32: 12, 64: 0, 128: 0}      # the narrowest covering B
    plain.close()
    cache = T.TuneCache(str(tmp_path / "t.json"))
    gpu = torch.cuda.get_device_name(0)
    cache.put(gpu, T.batch_key_for(s.n, 20, "fp32"), {"batch_tc": 1, "batch_bn": 128}, 0.1)
    tuned = BatchPlan([s], [b], [u], tune_cache=cache)
    assert tuned.info()["tc_items_bn"] == {32: 0, 64: 0, 128: 12}
    tuned.close()
    # a real tuning pass picks one of the candidates and leaves it on the solver
    best, ms = T.tune_batch(s, b, u, sweeps=2, cache=cache, save=False)
    assert ms > 0 and all(s.get_tuning()[k] == v for k, v in best.items())
