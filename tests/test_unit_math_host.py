"""The path kernel's own FP32 functions (sdd_mc.cu), checked on the host.

- log_unit: its polynomial coefficients are the ones fit_log_unit.py derives (a weighted
  least-squares fit of (log1p f - f) / f^2, rounded to FP32), and the kernel's sequence of
  operations, emulated with exactly rounded FP32 fused multiply-adds, stays within 1 ulp of the
  logarithm over a sample of the uniforms the kernel draws.
- sincos_2pi: its series coefficients are (pi/2)^n / n! rounded to FP32, and the emulated steps
  (quadrant reduction, paired series, sign bits) stay within 1 ulp of 1 of sin and cos of 2 pi u.

The GPU test checks both over all 2^23 uniforms on the device."""
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


def _kernel_source(signature="__device__ __forceinline__ float log_unit(float u)"):
    with open(os.path.join(CSRC, "sdd_mc.cu")) as f:
        src = f.read()
    body = src[src.index(signature):]
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


def _sincos_coefficients():
    """(sine, cosine) pairs of the paired Horner steps, in the order the kernel applies them."""
    body = _kernel_source("__device__ __forceinline__ void sincos_2pi(float u, float* sn, float* cs)")
    hexf = r"(-?0x[0-9a-fA-F.]+p[-+]?\d+)f"
    pairs = re.findall(r"make_float2\(" + hexf + r", " + hexf + r"\)", body)
    return [(float.fromhex(a), float.fromhex(b)) for a, b in pairs]


def test_sincos_coefficients_are_the_taylor_series():
    pairs = _sincos_coefficients()
    # first pair: the leading (degree 9, degree 10) coefficients, then one pair per step down to
    # (pi/2, -(pi/2)^2 / 2)
    sine_deg = [9, 7, 5, 3, 1]
    cos_deg = [10, 8, 6, 4, 2]
    assert len(pairs) == 5
    for (cs_, cc_), ds, dc in zip(pairs, sine_deg, cos_deg):
        want_s = (-1) ** ((ds - 1) // 2) * (math.pi / 2) ** ds / math.factorial(ds)
        want_c = (-1) ** (dc // 2) * (math.pi / 2) ** dc / math.factorial(dc)
        assert cs_ == _f32(want_s) and cc_ == _f32(want_c), (ds, dc)


def _sincos_2pi(u):
    """The kernel's steps: t = 4u, q = rint(t), r = t - q, the two series in r, quadrant swap and
    sign bits from q."""
    pairs = _sincos_coefficients()
    t = _f32(4.0 * u)
    q = float(round(t))  # Python rounds halves to even, as rintf
    qint = int(q)
    r = _f32(t - q)
    r2 = _f32(r * r)
    x, y = pairs[0]
    x, y = _fmaf(x, r2, pairs[1][0]), _fmaf(y, r2, pairs[1][1])
    for a, b in pairs[2:]:
        x, y = _fmaf(x, r2, a), _fmaf(y, r2, b)
    x, y = _fmaf(x, r, 0.0), _fmaf(y, r2, 1.0)
    s_, c_ = (y, x) if qint & 1 else (x, y)
    s_ = -s_ if (qint >> 1) & 1 else s_
    c_ = -c_ if ((qint + 1) >> 1) & 1 else c_
    return s_, c_


def test_emulated_kernel_sincos_within_one_ulp_of_one():
    rng = np.random.default_rng(20150402)
    m = list(rng.integers(0, 1 << 23, size=800))
    # quadrant boundaries (u near k/8 and k/4) and both ends
    for k in range(1, 8):
        c = round(k / 8 * (1 << 23) - 0.5)
        m += [c - 1, c, c + 1]
    m += [0, (1 << 23) - 1]
    tol = 2.0 ** -23
    for k in m:
        u = _f32(_f32(1.0 + k * 2.0 ** -23) - float.fromhex("0x1.fffffep-1"))
        s_, c_ = _sincos_2pi(u)
        assert abs(s_ - math.sin(2 * math.pi * u)) <= tol, (k, u, s_)
        assert abs(c_ - math.cos(2 * math.pi * u)) <= tol, (k, u, c_)
