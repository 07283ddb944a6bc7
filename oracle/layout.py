"""Interface nodes and subdomains of a Px x Py split -- oracle, TEST INFRASTRUCTURE.

The stochastic representation is evaluated only at the nodes of the artificial interfaces
between subdomains (Sec. 3.1, Sec. 3.5); every subdomain is then a Dirichlet problem whose
boundary is made of interface nodes and, where it touches it, the physical boundary.
"""
from __future__ import annotations

import numpy as np


def split_line(I, n, P):
    """Node index of the line that ends part I of an n-node direction split into P parts
    (part I spans split_line(I) .. split_line(I + 1); equal parts when P divides n - 1)."""
    return (I * (n - 1)) // P


def interface_nodes(nx, ny, px, py, periodic=0):
    """(M, 2) int array of (i, j) interface nodes in the canonical order.

    Vertical lines first (by increasing i, then j), then horizontal lines (by increasing j,
    then i), skipping nodes already listed on a vertical line.  Dirichlet: lines at
    i = floor(I (nx-1)/px) for I = 1..px-1, nodes j = 1..ny-2 (and the mirror for horizontal
    lines).  Periodic: lines at I = 0..px-1 (the line i = 0 is also i = nx-1), nodes
    j = 0..ny-2.  The position in this list is the node id used in the Philox counter.
    """
    if px > nx - 1 or py > ny - 1:
        raise ValueError("every subdomain must span at least one cell")
    vl = [split_line(I, nx, px) for I in (range(px) if periodic else range(1, px))]
    hl = [split_line(J, ny, py) for J in (range(py) if periodic else range(1, py))]
    if periodic:
        jr = range(0, ny - 1)
        ir = range(0, nx - 1)
    else:
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
    return [(split_line(I, nx, px), split_line(I + 1, nx, px), split_line(J, ny, py), split_line(J + 1, ny, py))
            for J in range(py) for I in range(px)]


def interface_sampling(nx, ny, px, py, periodic=0, stride=1, Lx=1.0, Ly=1.0):
    """Interface nodes evaluated by Monte Carlo, and the interpolation of the others (Sec. 3.6:
    the interface values may be evaluated at a sample of the nodes and interpolated elsewhere).

    Along every interface line the nodes whose index along the line is a multiple of `stride`,
    and the crossings with lines of the other direction, are sampled.  Any other node takes the
    linear interpolation, in its index along the line, between the nearest sampled node on
    either side; where there is none, the line's end takes its place: on a Dirichlet domain the
    boundary node there with its identity position, on a periodic domain the line's first node
    one period further on (its value plus (0, Ly) on a vertical line, (Lx, 0) on a horizontal one).

    Returns (sampled, fill): sampled is a bool array over the node list of interface_nodes;
    fill(est) returns a copy of est (M x 2) with every non-sampled row replaced by its
    interpolation of the sampled rows.
    """
    nodes = interface_nodes(nx, ny, px, py, periodic)
    M = len(nodes)
    if stride <= 1:
        return np.ones(M, dtype=bool), lambda est: np.array(est, dtype=np.float64, copy=True)
    ident = {(int(i), int(j)): m for m, (i, j) in enumerate(nodes)}
    vl = [split_line(I, nx, px) for I in (range(px) if periodic else range(1, px))]
    hl = [split_line(J, ny, py) for J in (range(py) if periodic else range(1, py))]
    sampled = np.zeros(M, dtype=bool)
    rules = []   # (m, weight of a, anchor a, anchor b); anchor = (node id or None, offset x, offset y)

    def line(points, crossing):
        # points: positions t = 0 .. L along the line, as (t, (i, j)) including both ends
        L = len(points) - 1
        anchors = {}
        for t, (i, j) in points:
            end = t == 0 or t == L
            if end and not periodic:
                anchors[t] = (None, Lx * i / (nx - 1), Ly * j / (ny - 1))
            elif end and t == L:        # periodic: the first node one period on
                i0, j0 = points[0][1]
                anchors[t] = (ident[(i0, j0)], Lx if i == nx - 1 and i0 == 0 else 0.0,
                              Ly if j == ny - 1 and j0 == 0 else 0.0)
            elif t % stride == 0 or crossing(i, j):
                anchors[t] = (ident[(i, j)], 0.0, 0.0)
        for t, (i, j) in points:
            if (i, j) not in ident or t in anchors:
                continue
            ta = max(u for u in anchors if u < t)
            tb = min(u for u in anchors if u > t)
            rules.append((ident[(i, j)], (tb - t) / (tb - ta), anchors[ta], anchors[tb]))

    for i in vl:
        pts = [(j, (i, j)) for j in range(ny)]
        line(pts, lambda a, b: b in hl)
    for j in hl:
        pts = [(i, (i, j)) for i in range(nx)]
        line(pts, lambda a, b: a in vl)
    interp = {m for m, _, _, _ in rules}
    sampled[:] = True
    for m in interp:
        sampled[m] = False

    def fill(est):
        out = np.array(est, dtype=np.float64, copy=True)
        def value(anchor):
            node, ox, oy = anchor
            base = np.zeros(2) if node is None else out[node]
            return np.array([base[0] + ox, base[1] + oy])
        for m, w, a, b in rules:
            out[m] = w * value(a) + (1.0 - w) * value(b)
        return out

    return sampled, fill
