"""Pins of the oracle's monitor evaluation and finite-difference gradient (Sec. 2, 3.4)."""
import numpy as np
import pytest

import workloads as W
from oracle.monitor import analytic_monitor, fd_gradient, monitor_on_grid, wrap_copy


def grid(nx, ny):
    xi = np.arange(nx) / (nx - 1)
    eta = np.arange(ny) / (ny - 1)
    return np.meshgrid(xi, eta)


@pytest.mark.parametrize("nx,ny", [(3, 3), (9, 13), (33, 33)])
def test_fd_gradient_exact_for_quadratics(nx, ny):
    """Central and one-sided second-order differences are exact for quadratics."""
    XI, ETA = grid(nx, ny)
    f = 1 + 2 * XI - 3 * ETA + 0.5 * XI ** 2 + 0.7 * XI * ETA - 1.3 * ETA ** 2
    gx, gy = fd_gradient(f, 0)
    assert np.allclose(gx, 2 + XI + 0.7 * ETA, atol=1e-11)
    assert np.allclose(gy, -3 + 0.7 * XI - 2.6 * ETA, atol=1e-11)


def test_fd_gradient_periodic_second_order():
    errs = []
    for n in (17, 33, 65):
        XI, ETA = grid(n, n)
        f = np.sin(2 * np.pi * XI) * np.cos(2 * np.pi * ETA)
        gx, gy = fd_gradient(f, 1)
        ex = 2 * np.pi * np.cos(2 * np.pi * XI) * np.cos(2 * np.pi * ETA)
        ey = -2 * np.pi * np.sin(2 * np.pi * XI) * np.sin(2 * np.pi * ETA)
        errs.append(max(np.abs(gx - ex).max(), np.abs(gy - ey).max()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_front_monitor_gradient_matches_numerical_derivative():
    """|grad u| of u = tanh(R (r - r0 - v t)) from a fine central difference of u itself."""
    alpha, R, r0, v, cx, cy = 50.0, 50.0, 0.25, 0.1, 0.5, 0.5
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, 400)
    y = rng.uniform(0, 1, 400)
    t = 0.37
    u = lambda a, b: np.tanh(R * (np.hypot(a - cx, b - cy) - r0 - v * t))
    h = 1e-6
    ux = (u(x + h, y) - u(x - h, y)) / (2 * h)
    uy = (u(x, y + h) - u(x, y - h)) / (2 * h)
    expect = np.sqrt(1 + alpha * (ux ** 2 + uy ** 2))
    got = analytic_monitor(W.MONITOR_FRONT, [alpha, R, r0, v, cx, cy], x, y, t)
    assert np.allclose(got, expect, rtol=1e-6)
    assert abs(analytic_monitor(W.MONITOR_FRONT, [alpha, R, r0, v, cx, cy],
                                np.array([0.5 + r0]), np.array([0.5]), 0.0)[0] - np.sqrt(1 + alpha * R * R)) < 1e-12


def test_gauss_and_bumps_values():
    a, b = 10.0, 50.0
    g = analytic_monitor(W.MONITOR_GAUSS, [a, b, 0.5, 0.5], np.array([0.5, 0.6]), np.array([0.5, 0.5]), 0.0)
    assert np.allclose(g, [np.sqrt(11.0), np.sqrt(1 + a * np.exp(-b * 0.01))])
    p = [3.0, 0.1, 0.2, 0.3, 5.0, 0.05, 0.7, 0.7]
    bm = analytic_monitor(W.MONITOR_BUMPS, p, np.array([0.2, 0.7, 0.0]), np.array([0.3, 0.7, 1.0]), 0.0)
    assert np.isclose(bm[0], 1 + 3.0 + 5.0 * np.exp(-(0.5 ** 2 + 0.4 ** 2) / 0.05 ** 2))
    assert np.isclose(bm[1], 1 + 5.0 + 3.0 * np.exp(-(0.5 ** 2 + 0.4 ** 2) / 0.01))
    assert np.ones(1) == analytic_monitor(W.MONITOR_BUMPS, [], np.zeros(1), np.zeros(1), 0.0)


def test_periodic_monitor_uses_minimum_image_and_wrap_copy():
    n = 17
    XI, ETA = grid(n, n)
    om = monitor_on_grid(W.MONITOR_GAUSS, [4.0, 20.0, 0.05, 0.95], XI, ETA, 0.0, periodic=1)
    raw = analytic_monitor(W.MONITOR_GAUSS, [4.0, 20.0, 0.05, 0.95], XI, ETA, 0.0, periodic=1)
    assert np.allclose(raw[:, -1], raw[:, 0], atol=1e-12)  # minimum image: xi = 1 is xi = 0
    # the bump near the corner is seen across the periodic boundary
    assert np.allclose(om[:, -1], om[:, 0]) and np.allclose(om[-1, :], om[0, :])
    far = analytic_monitor(W.MONITOR_GAUSS, [4.0, 20.0, 0.05, 0.95], np.array([0.95]), np.array([0.05]),
                           0.0, periodic=1)
    assert np.isclose(far[0], np.sqrt(1 + 4.0 * np.exp(-20.0 * (0.1 ** 2 + 0.1 ** 2))))
