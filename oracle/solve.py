"""Deterministic subdomain and single-domain solves -- oracle, TEST INFRASTRUCTURE.

Each subdomain is a Dirichlet problem for the mesh generator with the Monte Carlo values on
its artificial interfaces and the physical boundary values elsewhere (Sec. 3.5).  The
generator is discretised with centred differences in space; in time this project uses
backward Euler (the paper's forward Euler, Sec. 3.5, is unstable at these step sizes), so a
step solves, for every interior node P with neighbours E, W, N, S,

  form 0 (tau x_t = div(omega grad x)):
      x_P + r sum_nb a_nb (x_P - x_nb) = x^n_P
  form 1 (tau x_t = grad omega / omega . grad x + lap x, i.e. omega x_t = div(omega grad x)/tau):
      omega_P x_P + r sum_nb a_nb (x_P - x_nb) = omega_P x^n_P

with r = dt / tau, a_E = (omega_P + omega_E)/2 / h_xi^2 (face average), a_N the same with
h_eta.  The system is symmetric positive definite; the oracle solves it directly (SuperLU).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def box_system(omega, xn, i0, i1, j0, j1, dt, tau, form):
    """Matrix and right-hand-side builder for the interior of the node box [i0,i1] x [j0,j1].

    Returns (A, rhs_fn) where rhs_fn(rim, prev) gives the right-hand side for the rim values
    in `rim` (full grid array, only rim nodes read) and previous mesh `prev` (full grid array).
    """
    ny, nx = omega.shape
    hx2 = float(nx - 1) ** 2   # 1 / h_xi^2
    hy2 = float(ny - 1) ** 2   # 1 / h_eta^2
    r = dt / tau
    ii = list(range(i0 + 1, i1))
    jj = list(range(j0 + 1, j1))
    ni, nj = len(ii), len(jj)
    index = {}
    for b, j in enumerate(jj):
        for a, i in enumerate(ii):
            index[(i, j)] = b * ni + a
    rows, cols, vals = [], [], []
    rim_terms = []   # (row, (i, j) of rim neighbour, coefficient)
    diag_w = np.zeros(ni * nj)
    for (i, j), P in index.items():
        wP = omega[j, i]
        nbs = [((i + 1, j), 0.5 * (wP + omega[j, i + 1]) * hx2),
               ((i - 1, j), 0.5 * (wP + omega[j, i - 1]) * hx2),
               ((i, j + 1), 0.5 * (wP + omega[j + 1, i]) * hy2),
               ((i, j - 1), 0.5 * (wP + omega[j - 1, i]) * hy2)]
        d = wP if form == 1 else 1.0
        diag_w[P] = d
        for nb, a in nbs:
            d += r * a
            if nb in index:
                rows.append(P); cols.append(index[nb]); vals.append(-r * a)
            else:
                rim_terms.append((P, nb, r * a))
        rows.append(P); cols.append(P); vals.append(d)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(ni * nj, ni * nj))
    order = [None] * (ni * nj)
    for key, P in index.items():
        order[P] = key

    def rhs_fn(rim, prev):
        b = np.array([diag_w[P] * prev[j, i] for P, (i, j) in enumerate(order)])
        for P, (i, j), c in rim_terms:
            b[P] += c * rim[j, i]
        return b

    return A, rhs_fn, order


def solve_box(omega, rim_x, rim_y, xn, yn, i0, i1, j0, j1, dt, tau, form):
    """Backward-Euler solve of both mesh components on the interior of one node box.

    rim_x, rim_y: full-grid arrays holding the Dirichlet values on the box rim.
    xn, yn: the previous mesh (full grid).  Returns (x_int, y_int, order) with the interior
    values listed in `order` (a list of (i, j)).
    """
    A, rhs_fn, order = box_system(omega, xn, i0, i1, j0, j1, dt, tau, form)
    lu = spla.splu(A.tocsc())
    return lu.solve(rhs_fn(rim_x, xn)), lu.solve(rhs_fn(rim_y, yn)), order


def single_domain_step(omega, xn, yn, dt, tau, form, Lx=1.0, Ly=1.0):
    """One backward-Euler step on the whole Dirichlet domain (boundary mesh = identity).

    This is the single-domain reference mesh of the paper's quality comparison (Sec. 3.7)."""
    ny, nx = omega.shape
    xi = np.arange(nx) / (nx - 1)
    eta = np.arange(ny) / (ny - 1)
    bx = np.broadcast_to(Lx * xi[None, :], (ny, nx)).copy()
    by = np.broadcast_to(Ly * eta[:, None], (ny, nx)).copy()
    xs, ys, order = solve_box(omega, bx, by, xn, yn, 0, nx - 1, 0, ny - 1, dt, tau, form)
    out_x, out_y = bx.copy(), by.copy()
    for P, (i, j) in enumerate(order):
        out_x[j, i] = xs[P]
        out_y[j, i] = ys[P]
    return out_x, out_y


def periodic_single_domain_step(omega, xn, yn, dt, tau, form, Lx=1.0, Ly=1.0):
    """One backward-Euler step on the whole doubly periodic domain (no interfaces): the
    single-domain reference of the paper's periodic experiments (Sec. 4.2, Sec. 3.7).

    Unknowns are the (nx-1) x (ny-1) distinct nodes; a neighbour across the seam i = nx-1 is
    node 0 with x shifted by Lx (likewise y and Ly across j = ny-1), the direct-coordinate
    extension of Sec. 2.  Returns full-grid arrays including the wrap column and row."""
    ny, nx = omega.shape
    mx, my = nx - 1, ny - 1
    hx2 = float(nx - 1) ** 2
    hy2 = float(ny - 1) ** 2
    r = dt / tau
    n = mx * my
    idx = lambda i, j: (j % my) * mx + (i % mx)
    rows, cols, vals = [], [], []
    bx = np.zeros(n)
    by = np.zeros(n)
    for j in range(my):
        for i in range(mx):
            P = idx(i, j)
            wP = omega[j, i]
            d = wP if form == 1 else 1.0
            bx[P] = d * xn[j, i]
            by[P] = d * yn[j, i]
            diag = d
            for (di, dj, h2) in ((1, 0, hx2), (-1, 0, hx2), (0, 1, hy2), (0, -1, hy2)):
                ii, jj = i + di, j + dj
                a = r * 0.5 * (wP + omega[jj % my, ii % mx]) * h2
                diag += a
                rows.append(P); cols.append(idx(ii, jj)); vals.append(-a)
                # period offsets of the neighbour's coordinates across the seams
                bx[P] += a * Lx * (ii // mx)
                by[P] += a * Ly * (jj // my)
            rows.append(P); cols.append(P); vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)).tocsc()
    lu = spla.splu(A)
    sx, sy = lu.solve(bx), lu.solve(by)
    out_x = np.empty((ny, nx))
    out_y = np.empty((ny, nx))
    for j in range(ny):
        for i in range(nx):
            P = idx(i, j)
            out_x[j, i] = sx[P] + Lx * (i // mx)
            out_y[j, i] = sy[P] + Ly * (j // my)
    return out_x, out_y
