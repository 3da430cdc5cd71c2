"""The FP64 -> FP16 rounding the FP16 store and right-hand sides use
(csrc/f16_round.cuh) compiled for the host with g++: its 32-bit fast path
equals the general routine, and both equal numpy's float64 -> float16
conversion (round to nearest even, no double rounding) of v * 2^-k wherever
that is finite, with 65504 where it overflows (the routine saturates)."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r'''
#include <cstdint>
#include <cstdio>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double v) { long long r; std::memcpy(&r, &v, 8); return r; }
#include "f16_round.cuh"
int main() {
  double v; int k;
  while (std::scanf("%la %d", &v, &k) == 2)
    std::printf("%u %u\n", (unsigned)pide::f16_bits_scaled(v, k), (unsigned)pide::f16_bits_scaled_any(v, k));
  return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("f16")
    src = d / "f16.cpp"
    src.write_text(SHIM)
    exe = d / "f16"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_1602_00001_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def test_fast_path_equals_general_and_numpy(prog):
    rng = np.random.default_rng(11)
    k = rng.integers(-40, 40, 20000)
    v = rng.standard_normal(20000) * 2.0 ** (k + rng.integers(-30, 18, 20000))
    # exact FP16 ties, one FP64 ulp either side, zeros, subnormals, huge values
    t = (1.0 + 2.0 ** -11) * 2.0 ** k[:200]
    v[:200] = t
    v[200:400] = np.nextafter(t, np.inf)
    v[400:600] = -np.nextafter(t, -np.inf)
    v[600:610] = 0.0
    v[610:620] = -0.0
    v[620:630] = 5e-324
    v[630:640] = 1e300
    inp = "\n".join(f"{x.hex()} {int(kk)}" for x, kk in zip(v, k))
    out = subprocess.run([prog], input=inp, capture_output=True, text=True, check=True).stdout.split()
    fast = np.array(out[0::2], dtype=np.uint16)
    gen = np.array(out[1::2], dtype=np.uint16)
    assert np.array_equal(fast, gen)
    scaled = v * 2.0 ** (-k.astype(np.float64))
    with np.errstate(over="ignore"):
        ref = scaled.astype(np.float16)
    ref = np.where(np.isinf(ref), np.copysign(np.float16(65504), scaled).astype(np.float16), ref)
    assert np.array_equal(fast, ref.view(np.uint16))
