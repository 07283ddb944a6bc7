"""Moving physical boundary -- oracle, TEST INFRASTRUCTURE.

Sec. 2: on the physical boundary the normal components stay fixed (x = 0 on xi = 0, x = Lx on
xi = 1, y = 0 on eta = 0, y = Ly on eta = 1); the tangential ones -- x along eta = 0 and eta = 1,
y along xi = 0 and xi = 1 -- follow the one-dimensional form of the mesh generator along their
side.  One step of it is the 1-D restriction of the subdomain step (backward Euler, centred
differences, face-averaged monitor, form 1 multiplied through by omega):

    d_k b_k + r sum_{nb = k +- 1} c_{k,nb} (b_k - b_nb) = d_k b^n_k,   k = 1 .. n-2,
    c_{k,k+1} = (omega_k + omega_{k+1}) / 2 / h^2,   d_k = 1 (form 0) or omega_k (form 1),

with the corner values b_0, b_{n-1} fixed.  The oracle solves each side's tridiagonal system
with a dense solver.
"""
from __future__ import annotations

import numpy as np


def side_step(w, b, r, form):
    """One backward-Euler step of the 1-D generator on one side: w, b the monitor and the
    tangential coordinate at the side's n nodes (ends fixed).  Returns the new b."""
    n = len(b)
    h2 = float(n - 1) ** 2
    out = np.array(b, dtype=np.float64, copy=True)
    if n <= 2:
        return out
    m = n - 2
    A = np.zeros((m, m))
    rhs = np.zeros(m)
    for k in range(1, n - 1):
        d = w[k] if form == 1 else 1.0
        cw = r * (0.5 * (w[k] + w[k - 1]) * h2)
        ce = r * (0.5 * (w[k] + w[k + 1]) * h2)
        row = k - 1
        A[row, row] = d + cw + ce
        rhs[row] = d * b[k]
        if k - 1 >= 1:
            A[row, row - 1] = -cw
        else:
            rhs[row] += cw * b[0]
        if k + 1 <= n - 2:
            A[row, row + 1] = -ce
        else:
            rhs[row] += ce * b[n - 1]
    out[1:n - 1] = np.linalg.solve(A, rhs)
    return out


def boundary_mesh_step(prob, omega, x, y):
    """New tangential boundary coordinates after one step, in the layout [x on eta = 0 (nx),
    x on eta = 1 (nx), y on xi = 0 (ny), y on xi = 1 (ny)]."""
    r = prob.dt / prob.tau
    nx, ny = prob.nx, prob.ny
    bottom = side_step(omega[0, :], x[0, :], r, prob.form)
    top = side_step(omega[ny - 1, :], x[ny - 1, :], r, prob.form)
    left = side_step(omega[:, 0], y[:, 0], r, prob.form)
    right = side_step(omega[:, nx - 1], y[:, nx - 1], r, prob.form)
    return np.concatenate([bottom, top, left, right])


def boundary_arrays(prob, bnd):
    """Full-grid boundary values (bx, by) of the new mesh from boundary_mesh_step's layout."""
    nx, ny = prob.nx, prob.ny
    bx = np.full((ny, nx), np.nan)
    by = np.full((ny, nx), np.nan)
    bottom, top = bnd[:nx], bnd[nx:2 * nx]
    left, right = bnd[2 * nx:2 * nx + ny], bnd[2 * nx + ny:]
    bx[0, :], by[0, :] = bottom, 0.0
    bx[ny - 1, :], by[ny - 1, :] = top, prob.Ly
    bx[:, 0], by[:, 0] = 0.0, left
    bx[:, nx - 1], by[:, nx - 1] = prob.Lx, right
    return bx, by
