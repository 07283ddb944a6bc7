"""The path kernel's FP32 logarithm (log_unit in sdd_mc.cu), checked on the host: its polynomial
coefficients are the ones fit_log_unit.py derives (a weighted least-squares fit of
(log1p f - f) / f^2, rounded to FP32), and the kernel's sequence of operations, emulated here with
exactly rounded FP32 fused multiply-adds, stays within 1 ulp of the logarithm over a sample of the
uniforms the kernel draws (the GPU test checks all 2^23 of them on the device)."""
import math
import os
import re
import struct
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1504_00084_gb300", "csrc")


def _kernel_source():
    with open(os.path.join(CSRC, "sdd_mc.cu")) as f:
        src = f.read()
    body = src[src.index("__device__ __forceinline__ float log_unit(float u)"):]
    return body[:body.index("\n}\n")]


def _coefficients_in_kernel():
    """The polynomial's constants, highest degree first, as the kernel's Horner steps use them."""
    body = _kernel_source()
    first = re.search(r"float p = (-?0x[0-9a-fA-F.]+p-?\d+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, f, (-?0x[0-9a-fA-F.]+p-?\d+)f\);", body)
    return [float.fromhex(v) for v in [first] + rest]


def test_coefficients_are_the_fit():
    pytest.importorskip("mpmath")
    sys.path.insert(0, CSRC)
    try:
        import fit_log_unit
    finally:
        sys.path.remove(CSRC)
    fitted = fit_log_unit.coefficients()          # constant term first
    assert _coefficients_in_kernel() == list(reversed(fitted))


def _f32(x):
    return float(np.float32(x))


def _fmaf(a, b, c):
    """FP32 fused multiply-add, rounded once (exact rational arithmetic, then one rounding)."""
    exact = Fraction(a) * Fraction(b) + Fraction(c)
    return _round_f32(exact)


def _round_f32(q):
    """Round a rational to the nearest FP32 value (ties to even); normal range only."""
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    q = abs(q)
    e = math.floor(math.log2(q.numerator) - math.log2(q.denominator))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scaled = q / Fraction(2) ** (e - 23)          # in [2^23, 2^24)
    n = scaled.numerator // scaled.denominator
    rem = scaled - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * float(Fraction(n) * Fraction(2) ** (e - 23))


def _bits(x):
    return struct.unpack("<i", struct.pack("<f", x))[0]


def _from_bits(i):
    return struct.unpack("<f", struct.pack("<i", i))[0]


def _log_unit(u):
    """The kernel's steps: exponent split at sqrt(1/2), Horner in f, f + f^2 P(f), then e ln 2 in
    two parts.  Products and sums outside an fmaf round to FP32 on their own."""
    coeffs = _coefficients_in_kernel()
    i = _bits(u)
    e = (i - 0x3F3504F3) >> 23
    f = _f32(_from_bits(i - (e << 23)) - 1.0)      # exact: a Sterbenz subtraction
    ef = float(e)
    p = coeffs[0]
    for c in coeffs[1:]:
        p = _fmaf(p, f, c)
    t = _fmaf(_f32(f * f), p, f)
    return _fmaf(ef, float.fromhex("0x1.62e430p-1"), _fmaf(ef, float.fromhex("-0x1.05c610p-29"), t))


def _ulp(x):
    x = abs(_f32(x))
    return _from_bits(_bits(x) + 1) - x


def test_emulated_kernel_logarithm_within_one_ulp():
    rng = np.random.default_rng(20150401)
    m = list(rng.integers(0, 1 << 23, size=1500))
    # both ends of the range, the split at sqrt(1/2) and the neighbourhood of 1
    m += [0, 1, 2, (1 << 23) - 1, (1 << 23) - 2, 5931642, 5931641, 5931643, (1 << 23) - 17, 1 << 22]
    for k in m:
        u = _f32(1.0 + k * 2.0 ** -23) - float.fromhex("0x1.fffffep-1")   # the kernel's uniform
        u = _f32(u)
        got = _log_unit(u)
        exact = math.log(u)
        assert abs(got - exact) <= _ulp(exact), (k, u, got, exact)
