"""Geometric mesh quality (Eq. 8) and the SD/SDD ratio of Sec. 3.7 -- oracle, TEST INFRASTRUCTURE.

Q(K) = tr(J^T J) / (2 sqrt(det J^T J)) for the Jacobian J of the map (xi, eta) -> (x, y) on
cell K; for a 2 x 2 Jacobian sqrt(det J^T J) = |det J|, and Q >= 1 with equality exactly for
a scaled rotation (a square cell).  The Jacobian of cell (i, j) is taken from its edges:
x_xi = the mean of the cell's two xi-edges, x_eta = the mean of its two eta-edges (the grid
spacing cancels in the ratio).
"""
from __future__ import annotations

import numpy as np


def cell_quality(x, y):
    """Q per cell, shape (ny-1, nx-1)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x_xi = 0.5 * ((x[:-1, 1:] - x[:-1, :-1]) + (x[1:, 1:] - x[1:, :-1]))
    y_xi = 0.5 * ((y[:-1, 1:] - y[:-1, :-1]) + (y[1:, 1:] - y[1:, :-1]))
    x_eta = 0.5 * ((x[1:, :-1] - x[:-1, :-1]) + (x[1:, 1:] - x[:-1, 1:]))
    y_eta = 0.5 * ((y[1:, :-1] - y[:-1, :-1]) + (y[1:, 1:] - y[:-1, 1:]))
    tr = x_xi ** 2 + y_xi ** 2 + x_eta ** 2 + y_eta ** 2
    det = np.abs(x_xi * y_eta - x_eta * y_xi)
    return 0.5 * tr / det


def ratio_stats(q_sd, q_sdd):
    """R(K) = Q_SD / Q_SDD per cell, its maximum and mean over the cells (Sec. 3.7), and the
    ratio of the extreme qualities max Q_SD / max Q_SDD."""
    r = np.asarray(q_sd) / np.asarray(q_sdd)
    return {"R_max": float(r.max()), "R_mean": float(r.mean()),
            "maxQ_ratio": float(np.max(q_sd) / np.max(q_sdd))}
