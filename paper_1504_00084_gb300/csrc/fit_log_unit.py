"""Coefficients of log_unit (sdd_mc.cu): the degree-8 polynomial P with
ln(1 + f) ~ f + f^2 P(f) on f in [sqrt(1/2) - 1, sqrt(2) - 1], fitted by weighted least squares
on 4000 Chebyshev nodes (weight |f| / |ln(1 + f)|: the error of f^2 P relative to ln(1 + f)),
with (ln(1 + f) - f) / f^2 evaluated in 40-digit arithmetic, then rounded to FP32.
Prints the coefficients from the constant term up, in C hexadecimal float notation.
Needs numpy and mpmath; not part of the build."""
import numpy as np
from mpmath import mp


def coefficients(deg=8, n=4000):
    mp.dps = 40
    a, b = np.sqrt(0.5) - 1 - 1e-7, np.sqrt(2) - 1 + 1e-7
    xs = np.array([(a + b) / 2 + (b - a) / 2 * np.cos(np.pi * (k + 0.5) / n) for k in range(n)])
    ys = np.array([float((mp.log1p(mp.mpf(x)) - mp.mpf(x)) / mp.mpf(x) ** 2) for x in xs])
    w = np.abs(xs) / np.abs(np.log1p(xs))
    V = np.vander(xs, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V * w[:, None], ys * w, rcond=None)
    return [float(np.float32(v)) for v in c]


if __name__ == "__main__":
    for v in coefficients():
        print(float(v).hex().replace("0000000p", "p") + "f")
