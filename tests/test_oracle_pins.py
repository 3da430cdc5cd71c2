"""Pins for two oracle functions that every GPU parity assertion leans on:
Eq. (6)'s relative error (``rel_error_eq6``) and the two-term e4m3 quantiser
of the FP8 hi + lo store (``quantize_rows_e4m3(M, True)``).

Each pin is a check against something other than the function itself: a
hand-computed value, Table 1's printed cells (``table1_row`` measures its
error through ``rel_error_eq6``), or an error bound that follows from the
e4m3 format (3 mantissa bits, subnormal quantum 2^-9, largest finite 448).
The last tests plant plausible mistakes in copies of the two functions and
check that the pins reject every copy, so a mistake of that kind in the
oracle cannot pass the CPU suite."""
import os

import numpy as np
import pytest

from oracle import pide_oracle as O


# ---------------------------------------------------------------- Eq. (6)

# Two columns (one right-hand side per row, as everywhere in the oracle).
# Column 0: largest |u*| = 4, worst error 0.2 at an entry of size 2 -> 0.05.
# Column 1: largest |u*| = 0.5, error 0.04 at that entry -> 0.08, the worst.
_EQ6_REF = np.array([[1.0, -4.0, 2.0], [0.5, 0.25, -0.1]])
_EQ6_NUM = np.array([[1.0, -4.0, 2.2], [0.46, 0.25, -0.1]])


def eq6_pin_failures(fn, table1=None):
    """Names of the Eq. (6) pins that ``fn`` fails (empty: all pass).

    ``table1`` (optional) returns Table 1's no-rounding cell for n = 11 when
    computed with ``fn``."""
    bad = []
    # the worst column is the one with the smaller |u*|: 0.04 / 0.5
    if abs(fn(_EQ6_NUM, _EQ6_REF) - 0.08) > 1e-15:
        bad.append("two columns")
    # one column given as a vector: max |u - u*| / max |u*| = 0.3 / 6
    if abs(fn(np.array([3.0, -5.7, 1.3]), np.array([3.0, -6.0, 1.0])) - 0.05) > 1e-15:
        bad.append("one column")
    # identical inputs give 0; the error does not depend on the overall scale
    if fn(_EQ6_REF, _EQ6_REF) != 0.0:
        bad.append("zero")
    if abs(fn(1e7 * _EQ6_NUM, 1e7 * _EQ6_REF) - 0.08) > 1e-15:
        bad.append("scale")
    if table1 is not None and abs(table1(fn) - 0.0107) > 0.00005:
        bad.append("Table 1")
    return bad


def _table1_n11(fn, monkeypatch):
    with monkeypatch.context() as m:
        m.setattr(O, "rel_error_eq6", fn)
        return O.table1_row(11, [None])[0]


def test_eq6_pins(monkeypatch):
    assert eq6_pin_failures(O.rel_error_eq6, lambda f: _table1_n11(f, monkeypatch)) == []


def test_table1_row_measures_through_eq6(monkeypatch):
    """Table 1's cells come out of rel_error_eq6 (so its 24 printed cells pin
    Eq. 6): a stand-in that records its calls sees one call per rounding."""
    calls = []
    real = O.rel_error_eq6

    def spy(a, r):
        calls.append((np.shape(a), np.shape(r)))
        return real(a, r)

    with monkeypatch.context() as m:
        m.setattr(O, "rel_error_eq6", spy)
        out = O.table1_row(11, [2, None])
    assert len(calls) == 2 and calls[0] == ((121,), (121,))
    assert abs(out[1] - 0.0107) <= 0.00005 and abs(out[0] - 0.0112) <= 0.00005


# ---------------------------------------------------------------- two-term e4m3


def _matrix():
    rng = np.random.default_rng(21)
    M = rng.standard_normal((24, 257)) * 10.0 ** rng.uniform(-6, 2, (24, 257))
    # row 3: exactly s * (e4m3 values) with its maximum 448 s, s = 2^-5
    grid = O.round_e4m3(rng.uniform(-448, 448, 257))
    grid[17] = 448.0
    M[3] = grid * 2.0 ** -5
    # row 9: small entries, many in e4m3's subnormal range after scaling
    M[9] = rng.standard_normal(257) * 1e-3
    M[9, 0] = 50.0
    return M


def e4m3x2_pin_failures(fn):
    """Names of the pins of the two-term quantiser that ``fn`` fails."""
    bad = []
    M = _matrix()
    s, hi, lo = fn(M, True)
    s1, hi1, lo1 = fn(M, False)
    approx = s[:, None] * (hi + lo)
    # hi's rounding leaves at most 2^-4 |x| (normal) or 2^-10 (subnormal) of
    # x = M / s; lo takes that remainder to 4 more bits: 2^-8 |x| + 2^-10,
    # plus the two float32 roundings of x and x - hi (2^-24 each)
    bound = (2.0 ** -8 + 2.0 ** -22) * np.abs(M) + 2.0 ** -10 * s[:, None]
    if not np.all(np.abs(M - approx) <= bound):
        bad.append("2^-8 bound")
    # lo really carries the remainder: where x = M / s >= 4 (so that the
    # remainder is mostly above e4m3's subnormal range) the median error falls
    # by more than 8x
    e_hi = np.abs(M - s[:, None] * hi)
    e_2 = np.abs(M - approx)
    nz = (e_hi > 0) & (np.abs(M) >= 4.0 * s[:, None])
    if not np.median(e_2[nz] / e_hi[nz]) < 1 / 8:
        bad.append("lo carries the remainder")
    # lo is an e4m3 value within a sixteenth of the range (28 = 448 / 16)
    if not (np.array_equal(O.round_e4m3(lo), lo) and np.all(np.abs(lo) <= 28.0)):
        bad.append("lo range")
    # each nonzero row's largest |hi| is the top of the e4m3 range
    if not np.all(np.max(np.abs(hi), axis=1) == 448.0):
        bad.append("hi range")
    # a row exact in e4m3 (after its power-of-two scale) has lo = 0
    if not (s[3] == 2.0 ** -5 and np.array_equal(s[3] * hi[3], M[3]) and not np.any(lo[3])):
        bad.append("exact row")
    # hi and the scales are those of the single-term store; its lo is zero
    if not (np.array_equal(s1, s) and np.array_equal(hi1, hi) and not np.any(lo1)):
        bad.append("single term")
    return bad


def test_e4m3x2_pins():
    assert e4m3x2_pin_failures(O.quantize_rows_e4m3) == []


# ---------------------------------------------------------------- planted mistakes


def _eq6_axis0(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    return float(np.max(np.max(np.abs(a - r), axis=0) / np.max(np.abs(r), axis=0)))


def _eq6_global(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    return float(np.max(np.abs(a - r)) / np.max(np.abs(r)))


def _eq6_pointwise(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    m = r != 0
    return float(np.max(np.abs(a - r)[m] / np.abs(r)[m]))


def _eq6_mean_over_columns(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    return float(np.mean(np.max(np.abs(a - r), axis=1) / np.max(np.abs(r), axis=1)))


def _eq6_swapped(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    return float(np.max(np.max(np.abs(a - r), axis=1) / np.max(np.abs(a), axis=1)))


def _eq6_two_norm(a, r):
    a, r = np.atleast_2d(a), np.atleast_2d(r)
    return float(np.max(np.linalg.norm(a - r, axis=1) / np.linalg.norm(r, axis=1)))


@pytest.mark.parametrize("mutant", [_eq6_axis0, _eq6_global, _eq6_pointwise,
                                    _eq6_mean_over_columns, _eq6_swapped, _eq6_two_norm])
def test_eq6_pins_reject_planted_mistakes(mutant, monkeypatch):
    assert eq6_pin_failures(mutant, lambda f: _table1_n11(f, monkeypatch)) != []


def _q2(lo_rule, scale_div=448.0):
    """A copy of the two-term quantiser with the lo term (or the scale) replaced."""
    def fn(M, two_terms):
        mx = np.max(np.abs(M), axis=1)
        s = O.round_fp32(np.where(mx > 0, mx / scale_div, 1.0))
        x = M * (1.0 / s)[:, None]
        hi = O.round_e4m3(O.round_fp32(x))
        lo = lo_rule(M, s, x, hi) if two_terms else np.zeros_like(hi)
        return s, hi, lo
    return fn


_Q2_MUTANTS = {
    "lo dropped": _q2(lambda M, s, x, hi: np.zeros_like(hi)),
    "lo sign": _q2(lambda M, s, x, hi: O.round_e4m3(O.round_fp32(hi - x))),
    "lo unscaled": _q2(lambda M, s, x, hi: O.round_e4m3(O.round_fp32(M - s[:, None] * hi))),
    "lo re-rounds x": _q2(lambda M, s, x, hi: O.round_e4m3(O.round_fp32(x)) - hi),
    "lo 3 bits": _q2(lambda M, s, x, hi: O.round_to_bits(O.round_fp32(x - hi), 3)),
    "scale 256": _q2(lambda M, s, x, hi: O.round_e4m3(O.round_fp32(x - hi)), 256.0),
    "lo of hi's error squared": _q2(lambda M, s, x, hi: O.round_e4m3(O.round_fp32((x - hi) * 2))),
}


@pytest.mark.parametrize("name", sorted(_Q2_MUTANTS))
def test_e4m3x2_pins_reject_planted_mistakes(name):
    assert e4m3x2_pin_failures(_Q2_MUTANTS[name]) != []


def test_golden_dir_exists(golden_dir):
    assert os.path.isdir(golden_dir)
