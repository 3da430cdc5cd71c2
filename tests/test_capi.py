"""The C ABI: the library builds, loads and exports every entry point that
include/pide.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import pide_oracle as O
from paper_1602_00001_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    from paper_1602_00001_gb300 import build
    build.build()
    return binding.load_library()


def test_header_declares_the_boundary():
    syms = binding.header_symbols()
    for name in ["pide_setup", "pide_apply", "pide_residual", "pide_apply_backward",
                 "pide_apply_batched", "pide_destroy"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    so = binding.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in binding.header_symbols() if s not in exported]
    assert not missing, missing
    for s in binding.header_symbols():
        assert hasattr(lib, s)


def test_status_strings_and_version(lib):
    assert lib.pide_version() == 1
    assert lib.pide_status_string(0) == b"ok"
    assert b"invalid" in lib.pide_status_string(1)


def test_setup_rejects_bad_grid_without_gpu(lib):
    """Argument checks happen on the host before any CUDA call."""
    h = ctypes.c_void_p()
    g = binding.Grid(2, 5, 0.1)
    assert lib.pide_setup(ctypes.byref(g), None, 2, None, ctypes.byref(h)) == 1
    g = binding.Grid(5, 5, -1.0)
    assert lib.pide_setup(ctypes.byref(g), None, 2, None, ctypes.byref(h)) == 1
    g = binding.Grid(5, 5, 0.25)
    assert lib.pide_setup(ctypes.byref(g), None, 9, None, ctypes.byref(h)) == 1
    assert not h.value
    assert lib.pide_apply(None, None, None, 1, 0, 0.0, None, None, None) == 1


def test_oracle_binary_rounding_pins():
    """round_bf16 / round_fp32 against torch's conversions on float32-exact
    inputs (where a conversion through float32 rounds once), plus ties."""
    import torch
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4000).astype(np.float32).astype(np.float64) * 10.0 ** rng.integers(-8, 8, 4000)
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), ref)
    y = rng.standard_normal(1000) * 1e3
    assert np.array_equal(O.round_fp32(y), y.astype(np.float32).astype(np.float64))
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert O.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert O.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_oracle_bf16_correction_pins():
    """Q + s C against M: each entry within half an e4m3 step of |M - Q| (2^-4
    relative) plus half the e4m3 subnormal quantum (2^-10 s); the correction
    cuts the median error of Q alone by more than 8x; a row already exact in
    BF16 has s = 1 and C = 0; C's entries stay inside the finite e4m3 range and
    the largest reaches 448 on every nonzero row."""
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 300)) * 10.0 ** rng.uniform(-6, 2, (40, 300))
    M[7] = O.round_bf16(M[7])
    Q, s, C = O.quantize_bf16_correction(M)
    err_q = np.abs(M - Q)
    err = np.abs(M - (Q + s[:, None] * C))
    assert np.all(err <= 2.0 ** -4 * err_q + 2.0 ** -10 * s[:, None] * (1 + 1e-12))
    assert np.median(err[err_q > 0] / err_q[err_q > 0]) < 1 / 8
    assert s[7] == 1.0 and not np.any(C[7])
    assert np.all(np.abs(C) <= 448)
    rows = [p for p in range(40) if p != 7]
    assert np.all(np.max(np.abs(C[rows]), axis=1) == 448)


def test_oracle_fp16_rounding_pins():
    """round_fp16 against torch's float16 conversion of float32 values (normal
    and subnormal range, ties), inside the finite range; saturation at 65504."""
    import torch
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(8000) * 10.0 ** rng.uniform(-9, 4.7, 8000)).astype(np.float32)
    x = np.clip(x, -65504, 65504).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(O.round_fp16(x), ref)
    assert O.round_fp16(np.array([1.0 + 2.0 ** -11]))[0] == 1.0              # tie to even
    assert O.round_fp16(np.array([1.0 + 3 * 2.0 ** -11]))[0] == 1.0 + 2.0 ** -9
    assert O.round_fp16(np.array([2.0 ** -25]))[0] == 0.0                     # tie at the bottom
    assert O.round_fp16(np.array([3 * 2.0 ** -25]))[0] == 2.0 ** -23
    assert O.round_fp16(np.array([7e4, -1e9]))[0] == 65504.0
    assert O.round_fp16(np.array([-1e9]))[0] == -65504.0


def test_oracle_fp16_rounding_direct_from_double():
    """round_fp16 rounds once, from the FP64 value (as the GPU's integer
    conversion does): it equals numpy's direct float64 -> float16 conversion,
    including values one FP64 ulp either side of an FP16 tie, where a detour
    through float32 would round twice."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal(100000) * 10.0 ** rng.uniform(-9, 4.7, 100000)
    x = x[np.abs(x) < 65504]
    assert np.array_equal(O.round_fp16(x), x.astype(np.float16).astype(np.float64))
    ties = np.array([1.0 + 2.0 ** -11, 3.0 + 1.5 * 2.0 ** -10, 2.0 ** -20 + 2.0 ** -25,
                     5 * 2.0 ** -16 + 2.0 ** -25])
    near = np.concatenate([ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf), -ties])
    assert np.array_equal(O.round_fp16(near), near.astype(np.float16).astype(np.float64))
    # the float32 detour differs on the ulp-above cases (a double-rounding witness)
    up = np.nextafter(ties[:1], np.inf)
    assert O.round_fp16(up)[0] == 1.0 + 2.0 ** -10
    assert O.round_fp16(O.round_fp32(up))[0] == 1.0


def test_oracle_fp16_store_pins():
    """Power-of-two row scales put each row's maximum in [2^14, 2^15); s Q is
    within half an FP16 step of M (2^-11 relative) for entries above 2^-14 s;
    an all-zero row has s = 1; column scales put maxima in [2^11, 2^12); the
    correction term cuts the store's median error by more than 8x."""
    rng = np.random.default_rng(4)
    M = rng.standard_normal((30, 200)) * 10.0 ** rng.uniform(-7, 1, (30, 200))
    M[5] = 0.0
    s, Q = O.quantize_rows_fp16(M)
    assert np.all(np.log2(s) == np.round(np.log2(s)))
    mq = np.max(np.abs(Q), axis=1)
    rows = [p for p in range(30) if p != 5]
    assert np.all((mq[rows] >= 2 ** 14) & (mq[rows] <= 2 ** 15)) and s[5] == 1.0
    err = np.abs(M - s[:, None] * Q)
    normal = np.abs(M) >= 2.0 ** -14 * s[:, None]
    assert np.all(err[normal] <= 2.0 ** -11 * np.abs(M[normal]))
    t, R = O.quantize_cols_fp16(M[rows])
    mr = np.max(np.abs(R), axis=1)
    assert np.all((mr >= 2 ** 11) & (mr <= 2 ** 12))
    s2, Q2, c, C = O.quantize_fp16_correction(M[rows])
    e1 = np.abs(M[rows] - s2[:, None] * Q2)
    e2 = np.abs(M[rows] - s2[:, None] * Q2 - c[:, None] * C)
    nz = e1 > 0
    assert np.median(e2[nz] / e1[nz]) < 1 / 8


def test_oracle_e4m3_rounding_pins():
    """round_e4m3 against torch's float8_e4m3fn conversion of float32 values
    (normal and subnormal range, ties), inside the finite range."""
    import torch
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(6000) * 10.0 ** rng.uniform(-4, 2.6, 6000)).astype(np.float32)
    x = np.clip(x, -448, 448).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.round_e4m3(x), ref)
    # exact grid points and halfway cases: 1.0625 is halfway between 1 and 1.125 -> 1
    assert O.round_e4m3(np.array([1.0625]))[0] == 1.0
    assert O.round_e4m3(np.array([1.1875]))[0] == 1.25
    assert O.round_e4m3(np.array([2.0 ** -10]))[0] == 0.0          # ties to even at the bottom
    assert O.round_e4m3(np.array([3 * 2.0 ** -10]))[0] == 2.0 ** -8


def _header_enum(name):
    """{enumerator: value} of `typedef enum {...} name;` in include/pide.h."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "pide.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\}\s*" + name + ";", src).group(1)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"(PIDE_\w+)\s*=\s*(\d+)", body)}


def test_binding_precisions_and_tuning_keys_match_the_header():
    """The binding's precision names and tuning keys carry the header's values."""
    from paper_1602_00001_gb300 import binding
    prec = _header_enum("pide_precision")
    assert {("PIDE_" + k.upper()): v for k, v in binding.PRECISIONS.items()} == prec
    keys = _header_enum("pide_tune_key")
    assert {("PIDE_TUNE_" + k.upper()): v for k, v in binding.Solver.TUNE_KEYS.items()} == keys


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures carry the header's field offsets and sizes (a C
    program compiled against include/pide.h prints them)."""
    import os
    import subprocess
    from paper_1602_00001_gb300 import binding
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"pide_info": binding.Info, "pide_handle_info": binding.HandleInfo,
               "pide_auto_candidate": binding.AutoCandidate,
               "pide_auto_report": binding.AutoReport, "pide_grid": binding.Grid,
               "pide_grid3": binding.Grid3, "pide_profile": binding.Profile}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pide.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, value = line.split()
        cls = structs[cname]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (cname, field, got, value)
