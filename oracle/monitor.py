"""Monitor (mesh density) and its finite-difference gradient -- oracle, TEST INFRASTRUCTURE.

The monitor omega is evaluated on the current physical mesh at time t^n and then frozen for
the step (the alternating MP procedure, Sec. 2 and Sec. 3.2).  Its gradient with respect to
the computational coordinates is approximated by finite differences (Sec. 3.4).
"""
from __future__ import annotations

import numpy as np

from workloads import MONITOR_BUMPS, MONITOR_FRONT, MONITOR_GAUSS, MONITOR_NODAL, MONITOR_RINGS


def _offsets(x, y, cx, cy, periodic, Lx, Ly):
    dx = x - cx
    dy = y - cy
    if periodic:
        # minimum image on the periodic rectangle
        dx = dx - Lx * np.floor(dx / Lx + 0.5)
        dy = dy - Ly * np.floor(dy / Ly + 0.5)
    return dx, dy


def analytic_monitor(kind, params, x, y, t, periodic=0, Lx=1.0, Ly=1.0):
    """omega at the points (x, y) at time t, in FP64 (pointwise; see monitor_on_grid).

    GAUSS  (a, b, cx, cy):             sqrt(1 + a exp(-b |x - c|^2))
    FRONT  (alpha, R, r0, v, cx, cy):  sqrt(1 + alpha |grad u|^2) with u = tanh(R (r - r0 - v t)),
                                       r = |x - c|, so |grad u| = R (1 - u^2)  (the arc-length
                                       monitor of Sec. 1 / Sec. 4.1 for an analytic u)
    BUMPS  (a_1, w_1, cx_1, cy_1, ...): 1 + sum_i a_i exp(-|x - c_i|^2 / w_i^2)
    RINGS  (alpha, R, r2, cx_1, cy_1, ...): sqrt(1 + alpha |grad u|^2) with
                                       u = sum_k tanh(R (|x - c_k|^2 - r2))  (the five-ring
                                       problem of Sec. 4.2), grad u = sum_k R (1 - u_k^2) 2 (x - c_k)
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    params = [float(v) for v in params]
    if kind == MONITOR_GAUSS:
        a, b, cx, cy = params
        dx, dy = _offsets(x, y, cx, cy, periodic, Lx, Ly)
        om = np.sqrt(1.0 + a * np.exp(-b * (dx * dx + dy * dy)))
    elif kind == MONITOR_FRONT:
        alpha, R, r0, v, cx, cy = params
        dx, dy = _offsets(x, y, cx, cy, periodic, Lx, Ly)
        r = np.sqrt(dx * dx + dy * dy)
        u = np.tanh(R * (r - r0 - v * t))
        g = R * (1.0 - u * u)
        om = np.sqrt(1.0 + alpha * g * g)
    elif kind == MONITOR_BUMPS:
        om = np.ones_like(x)
        for q in range(len(params) // 4):
            a, w, cx, cy = params[4 * q:4 * q + 4]
            dx, dy = _offsets(x, y, cx, cy, periodic, Lx, Ly)
            om = om + a * np.exp(-(dx * dx + dy * dy) / (w * w))
    elif kind == MONITOR_RINGS:
        alpha, R, r2 = params[:3]
        gx = np.zeros_like(x)
        gy = np.zeros_like(x)
        for q in range(3, len(params) - 1, 2):
            dx, dy = _offsets(x, y, params[q], params[q + 1], periodic, Lx, Ly)
            uk = np.tanh(R * (dx * dx + dy * dy - r2))
            f = R * (1.0 - uk * uk) * 2.0
            gx = gx + f * dx
            gy = gy + f * dy
        om = np.sqrt(1.0 + alpha * (gx * gx + gy * gy))
    else:
        raise ValueError(f"unknown analytic monitor kind {kind}")
    return om


def monitor_on_grid(kind, params, x, y, t, periodic=0, Lx=1.0, Ly=1.0):
    """omega at the nodes of the current mesh; periodic grids copy node 0 onto the wrap node."""
    om = analytic_monitor(kind, params, x, y, t, periodic, Lx, Ly)
    return wrap_copy(om) if periodic else om


def wrap_copy(f):
    """Periodic grids store the wrap column/row: node (nx-1, j) is node (0, j), (i, ny-1) is (i, 0)."""
    f = np.array(f, dtype=np.float64, copy=True)
    f[:, -1] = f[:, 0]
    f[-1, :] = f[0, :]
    return f


def fd_gradient(om, periodic=0):
    """(d omega/d xi, d omega/d eta) at the nodes by finite differences (Sec. 3.4).

    Interior: central differences (f_{i+1} - f_{i-1}) (n-1)/2.
    Dirichlet boundary: one-sided second order (-3 f_0 + 4 f_1 - f_2) (n-1)/2 and its mirror.
    Periodic: central differences with wrapped neighbours (node n-1 is node 0).
    Arrays are row-major (ny, nx): axis 1 is xi, axis 0 is eta.
    """
    om = np.asarray(om, dtype=np.float64)
    return _fd_axis(om, 1, periodic), _fd_axis(om, 0, periodic)


def _fd_axis(f, axis, periodic):
    g = np.moveaxis(f, axis, 0)
    n = g.shape[0]
    c = 0.5 * (n - 1)
    d = np.empty_like(g)
    if periodic:
        m = n - 1  # distinct nodes 0..n-2
        for i in range(m):
            d[i] = (g[(i + 1) % m] - g[(i - 1) % m]) * c
        d[n - 1] = d[0]
    else:
        for i in range(1, n - 1):
            d[i] = (g[i + 1] - g[i - 1]) * c
        d[0] = (-3.0 * g[0] + 4.0 * g[1] - g[2]) * c
        d[n - 1] = (3.0 * g[n - 1] - 4.0 * g[n - 2] + g[n - 3]) * c
    return np.moveaxis(d, 0, axis)
