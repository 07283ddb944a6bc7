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

The paper's own local solver is forward Euler (Sec. 3.5), offered as an option: the same
operator applied explicitly in S substeps of dt / S, with S = ceil(max_P sum_nb r a_nb / d_P) --
the smallest count for which every substep is a convex combination of the node and its
neighbours (discrete maximum principle) -- and the rim values interpolated linearly in time
between the previous mesh and the new Dirichlet data.
"""
from __future__ import annotations

import math

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


def fe_substeps(c_sum_over_d):
    """Forward-Euler substeps for the largest sum_nb c_nb / d_P of a box: S = ceil(that), >= 1."""
    return max(1, int(math.ceil(c_sum_over_d)))


def solve_box_fe(omega, rim_x, rim_y, xn, yn, i0, i1, j0, j1, dt, tau, form):
    """Forward-Euler update of the interior of one node box (the paper's local solver, Sec. 3.5).

    rim_x, rim_y hold the new Dirichlet values on the box rim, xn, yn the previous mesh.  Every
    substep m = 0..S-1 moves each interior node by (1 / (S d_P)) sum_nb c_nb (x_nb - x_P), with
    rim neighbours at xn + (m / S)(rim - xn).  Returns (x_int, y_int, order, S) as solve_box."""
    ny, nx = omega.shape
    hx2 = float(nx - 1) ** 2
    hy2 = float(ny - 1) ** 2
    r = dt / tau
    ii = np.arange(i0 + 1, i1)
    jj = np.arange(j0 + 1, j1)
    order = [(i, j) for j in jj for i in ii]
    if len(order) == 0:
        return np.zeros(0), np.zeros(0), order, 1
    J, I = np.meshgrid(jj, ii, indexing="ij")
    w = omega[J, I]
    cE = r * (0.5 * (w + omega[J, I + 1]) * hx2)
    cW = r * (0.5 * (w + omega[J, I - 1]) * hx2)
    cN = r * (0.5 * (w + omega[J + 1, I]) * hy2)
    cS = r * (0.5 * (w + omega[J - 1, I]) * hy2)
    d = w if form == 1 else np.ones_like(w)
    S = fe_substeps(float(((cE + cW + cN + cS) / d).max()))
    ax = xn[j0:j1 + 1, i0:i1 + 1].astype(np.float64).copy()
    ay = yn[j0:j1 + 1, i0:i1 + 1].astype(np.float64).copy()
    px, py = xn[j0:j1 + 1, i0:i1 + 1], yn[j0:j1 + 1, i0:i1 + 1]
    qx, qy = rim_x[j0:j1 + 1, i0:i1 + 1], rim_y[j0:j1 + 1, i0:i1 + 1]
    rim = np.ones(ax.shape, bool)
    rim[1:-1, 1:-1] = False
    for m in range(S):
        f = m / S
        for a, p, q in ((ax, px, qx), (ay, py, qy)):
            a[rim] = p[rim] + f * (q[rim] - p[rim])
        for a in (ax, ay):
            c = a[1:-1, 1:-1]
            s_ = (cE * (a[1:-1, 2:] - c) + cW * (a[1:-1, :-2] - c)) + cN * (a[2:, 1:-1] - c) + cS * (a[:-2, 1:-1] - c)
            a[1:-1, 1:-1] = c + s_ / (S * d)
    return ax[1:-1, 1:-1].ravel(), ay[1:-1, 1:-1].ravel(), order, S


def periodic_single_domain_step_fe(omega, xn, yn, dt, tau, form, Lx=1.0, Ly=1.0):
    """Forward-Euler counterpart of periodic_single_domain_step: S substeps of the same
    operator on the doubly periodic grid (neighbours across a seam carry the period offset)."""
    ny, nx = omega.shape
    mx, my = nx - 1, ny - 1
    hx2 = float(nx - 1) ** 2
    hy2 = float(ny - 1) ** 2
    r = dt / tau
    w = omega[:my, :mx]
    wE, wW = np.roll(w, -1, axis=1), np.roll(w, 1, axis=1)
    wN, wS = np.roll(w, -1, axis=0), np.roll(w, 1, axis=0)
    cE = r * (0.5 * (w + wE) * hx2)
    cW = r * (0.5 * (w + wW) * hx2)
    cN = r * (0.5 * (w + wN) * hy2)
    cS = r * (0.5 * (w + wS) * hy2)
    d = w if form == 1 else np.ones_like(w)
    S = fe_substeps(float(((cE + cW + cN + cS) / d).max()))
    x = xn[:my, :mx].astype(np.float64).copy()
    y = yn[:my, :mx].astype(np.float64).copy()
    for _ in range(S):
        xE = np.roll(x, -1, axis=1); xE[:, -1] += Lx
        xW = np.roll(x, 1, axis=1); xW[:, 0] -= Lx
        x_new = x + ((cE * (xE - x) + cW * (xW - x)) + cN * (np.roll(x, -1, axis=0) - x) +
                     cS * (np.roll(x, 1, axis=0) - x)) / (S * d)
        yN = np.roll(y, -1, axis=0); yN[-1, :] += Ly
        yS = np.roll(y, 1, axis=0); yS[0, :] -= Ly
        y_new = y + ((cE * (np.roll(y, -1, axis=1) - y) + cW * (np.roll(y, 1, axis=1) - y)) + cN * (yN - y) +
                     cS * (yS - y)) / (S * d)
        x, y = x_new, y_new
    out_x = np.empty((ny, nx))
    out_y = np.empty((ny, nx))
    out_x[:my, :mx] = x
    out_y[:my, :mx] = y
    out_x[:my, mx] = x[:, 0] + Lx
    out_y[:my, mx] = y[:, 0]
    out_x[my, :] = out_x[0, :]
    out_y[my, :] = out_y[0, :] + Ly
    return out_x, out_y
