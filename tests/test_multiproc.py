"""The N > 1 host path of bench.py (replicas, no data-path collective):
max-over-ranks timing and the whole-job rate, with world_size 2 over gloo on
the CPU; the reference arm prints only on rank 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    mx = bench.reduce_max(ms, dist)
    rate = bench.whole_job_rate(world, 1024, 20, mx)
    dist.barrier()
    q.put((rank, mx, rate))
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, rate in out:
        assert mx == 150.0
        assert rate == pytest.approx(2 * 1024 * 20 / 0.150)


def test_reference_arm_silent_off_rank0(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.reference_arm(A()) == 0
    assert buf.getvalue() == ""


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5, None) == 3.5
