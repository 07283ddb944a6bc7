"""Interface nodes and subdomains of a Px x Py split -- oracle, TEST INFRASTRUCTURE.

The stochastic representation is evaluated only at the nodes of the artificial interfaces
between subdomains (Sec. 3.1, Sec. 3.5); every subdomain is then a Dirichlet problem whose
boundary is made of interface nodes and, where it touches it, the physical boundary.
"""
from __future__ import annotations

import numpy as np


def interface_nodes(nx, ny, px, py, periodic=0):
    """(M, 2) int array of (i, j) interface nodes in the canonical order.

    Vertical lines first (by increasing i, then j), then horizontal lines (by increasing j,
    then i), skipping nodes already listed on a vertical line.  Dirichlet: lines at
    i = I (nx-1)/px for I = 1..px-1, nodes j = 1..ny-2 (and the mirror for horizontal
    lines).  Periodic: lines at I = 0..px-1 (the line i = 0 is also i = nx-1), nodes
    j = 0..ny-2.  The position in this list is the node id used in the Philox counter.
    """
    if (nx - 1) % px or (ny - 1) % py:
        raise ValueError("grid intervals must divide evenly into subdomains")
    sx, sy = (nx - 1) // px, (ny - 1) // py
    if periodic:
        vl = [I * sx for I in range(px)]
        hl = [J * sy for J in range(py)]
        jr = range(0, ny - 1)
        ir = range(0, nx - 1)
    else:
        vl = [I * sx for I in range(1, px)]
        hl = [J * sy for J in range(1, py)]
        jr = range(1, ny - 1)
        ir = range(1, nx - 1)
    out = []
    for i in vl:
        for j in jr:
            out.append((i, j))
    vset = set(vl)
    for j in hl:
        for i in ir:
            if i not in vset:
                out.append((i, j))
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def subdomains(nx, ny, px, py):
    """List of (i0, i1, j0, j1): subdomain (I, J) spans nodes i0..i1, j0..j1 (rims included)."""
    sx, sy = (nx - 1) // px, (ny - 1) // py
    return [(I * sx, (I + 1) * sx, J * sy, (J + 1) * sy) for J in range(py) for I in range(px)]
