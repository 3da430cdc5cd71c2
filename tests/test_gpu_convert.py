"""The library's integer-pipe IEEE conversions (binary64 -> bfloat16 with
round-to-nearest-even, binary32 -> binary64) against CUDA's, bit for bit."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_conversions_match_cuda_bitwise():
    from paper_1602_00001_gb300 import build, binding
    build.build()
    lib = binding.load_library()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000) * 10.0 ** rng.uniform(-45, 45, 200000)
    # exact halfway cases between bfloat16 neighbours, both parities, and specials
    base = rng.standard_normal(2000).astype(np.float32).view(np.uint32) & 0xFFFF0000
    halves = (base.astype(np.uint64) << 32).view(np.float64) + 0.0
    halves = np.concatenate([halves * (1 + 2.0 ** -8), halves * (1 + 3 * 2.0 ** -8)])
    special = np.array([0.0, -0.0, 1.0, -1.0, 3.4e38, 3.4028235e38, 3.41e38, 1e-38, 1.1754943508222875e-38,
                        1e-39, 1e-45, 5e-324, np.inf, -np.inf, 1e300, -1e-300])
    x = np.concatenate([x, halves, special])
    f = np.concatenate([rng.standard_normal(100000).astype(np.float32) *
                        np.float32(10.0) ** rng.uniform(-40, 38, 100000).astype(np.float32),
                        np.array([0.0, -0.0, 1e-40, -1e-45, np.inf, 3.4e38], dtype=np.float32)])
    n = min(len(x), len(f))
    xd = torch.from_numpy(x[:n]).cuda()
    fd = torch.from_numpy(f[:n].astype(np.float32)).cuda()
    bm = torch.empty(n, dtype=torch.int16, device="cuda")
    bc = torch.empty_like(bm)
    dm = torch.empty(n, dtype=torch.float64, device="cuda")
    dc = torch.empty_like(dm)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.pide_selftest_convert(P(xd), P(fd), n, P(bm), P(bc), P(dm), P(dc), None)
    assert st == 0
    torch.cuda.synchronize()
    assert torch.equal(bm, bc)
    assert torch.equal(dm.view(torch.int64), dc.view(torch.int64))
