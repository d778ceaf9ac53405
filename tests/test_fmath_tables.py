"""The constant tables of the device's table-driven float64 log, log1p, exp
and expm1 (paper_2305_07181_gb300/csrc/fmath_tables.h, after Tang, ACM TOMS
1989/1990): the committed header is what its generator writes, and every
entry is checked against an independent 60-digit evaluation (mpmath):
ln(j/128) and 2^(j/32) as hi + lo pairs to ~2^-100, 1/c_j rounded to nearest,
ln 2 and ln 2 / 32 split with at most 36 significant bits in the high part and
the remainder rounded to nearest in the low part,
and the Taylor coefficients (-1)^(k+1)/k and 1/k! rounded to nearest."""
import importlib.util
import math
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2305_07181_gb300", "csrc")


def _header():
    with open(os.path.join(CSRC, "fmath_tables.h")) as f:
        return f.read()


def _scalar(text, name):
    m = re.search(rf"constexpr (?:double|int) {name} = ([^;,]+)[;,]", text)
    return float(m.group(1))


def _array(text, name):
    m = re.search(rf"{name}\[(\d+)\] = \{{(.*?)\}};", text, re.S)
    vals = [float(v) for v in m.group(2).replace("\n", " ").split(",") if v.strip()]
    assert len(vals) == int(m.group(1))
    return vals


def test_header_is_the_generator_output():
    spec = importlib.util.spec_from_file_location("gen_fmath_tables", os.path.join(CSRC, "gen_fmath_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.render() == _header()


def _rounded(x):
    """x (mpmath) rounded to the nearest float64."""
    return float(mpmath.mpf(x))


def test_log_and_exp_tables_against_60_digits():
    mpmath.mp.dps = 60
    h = _header()
    j0 = int(_scalar(h, "LOG_J0"))
    hi, lo, inv = _array(h, "LOG_C_HI"), _array(h, "LOG_C_LO"), _array(h, "LOG_INV_C")
    for t, (a, b, c) in enumerate(zip(hi, lo, inv)):
        j = j0 + t
        exact = mpmath.log(mpmath.mpf(j) / 128)
        assert a == _rounded(exact)
        assert abs(mpmath.mpf(a) + mpmath.mpf(b) - exact) <= mpmath.mpf(2) ** -100
        assert c == _rounded(mpmath.mpf(128) / j)
    eh, el = _array(h, "EXP_T_HI"), _array(h, "EXP_T_LO")
    for j, (a, b) in enumerate(zip(eh, el)):
        exact = mpmath.power(2, mpmath.mpf(j) / 32)
        assert a == _rounded(exact)
        assert abs(mpmath.mpf(a) + mpmath.mpf(b) - exact) <= mpmath.mpf(2) ** -100


def test_ln2_splits_and_coefficients():
    mpmath.mp.dps = 60
    h = _header()
    ln2 = mpmath.log(2)
    for hi_name, lo_name, exact in (("LN2_HI", "LN2_LO", ln2), ("L32_HI", "L32_LO", ln2 / 32)):
        a, b = _scalar(h, hi_name), _scalar(h, lo_name)
        m, _ = math.frexp(a)
        assert (m * 2 ** 36).is_integer()  # at most 36 significant bits: k ln2_hi exact for |k| < 2^17
        assert b == _rounded(exact - mpmath.mpf(a))  # the remainder, rounded to nearest
    assert _scalar(h, "INV_L32") == _rounded(32 / ln2)
    for k in range(2, 13):
        assert _scalar(h, f"LOG_C{k}") == _rounded(mpmath.mpf((-1) ** (k + 1)) / k)
    for k in range(2, 14):
        assert _scalar(h, f"EXP_E{k}") == _rounded(1 / mpmath.factorial(k))
