"""Monte Carlo evaluation of the stochastic representation at interface nodes -- oracle,
TEST INFRASTRUCTURE.

Each interface node's new mesh position is the expectation of Eq. (5a) (Dirichlet) or
Eq. (6) (periodic) over paths of the SDE of Eq. (5b) stepped by Eq. (7); it is estimated by
the arithmetic mean of N paths (Sec. 3.4).  The per-path work runs in the C core
(sdd_oracle.c); this module prepares its inputs and forms the estimates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _clib
from .monitor import fd_gradient

ADAPTIVE_GRANULE = 1024   # adaptive chunk totals are multiples of this many paths
ADAPTIVE_SAFETY = 1.03    # over-provisioning factor of the next chunk


@dataclass
class PathInputs:
    """Everything a path needs, in the working precision (float64 or float32)."""
    real: type
    struct: object
    keep: tuple  # arrays referenced by the struct


def prepare(prob, x, y, omega, tstep: int, real=np.float64, bnd=None) -> PathInputs:
    """Pack the frozen monitor, its FD gradient and the mesh displacement for the C core.

    The monitor and its gradient are computed in FP64 and rounded once to the working
    precision; so is the displacement X = x - Lx xi, Y = y - Ly eta of the previous mesh, and
    the new boundary mesh bnd of a moving boundary (oracle.boundary layout; None: identity).
    """
    real = np.dtype(real).type
    wxi, weta = fd_gradient(omega, prob.periodic)
    xi = np.arange(prob.nx, dtype=np.float64) / (prob.nx - 1)
    eta = np.arange(prob.ny, dtype=np.float64) / (prob.ny - 1)
    X = np.asarray(x, dtype=np.float64) - prob.Lx * xi[None, :]
    Y = np.asarray(y, dtype=np.float64) - prob.Ly * eta[:, None]
    arrs = tuple(np.ascontiguousarray(a, dtype=real) for a in (omega, wxi, weta, X, Y))
    if bnd is not None:
        arrs = arrs + (np.ascontiguousarray(bnd, dtype=real),)
    ct = _clib.ctypes.c_float if real is np.float32 else _clib.ctypes.c_double
    S = _clib.ProblemF32 if real is np.float32 else _clib.ProblemF64
    seed = int(prob.seed) & 0xFFFFFFFFFFFFFFFF
    s = S(nx=prob.nx, ny=prob.ny, periodic=prob.periodic, form=prob.form, K=prob.substeps,
          bicubic=prob.bicubic, bb_test=prob.bb_test, tstep=int(tstep),
          key0=seed & 0xFFFFFFFF, key1=seed >> 32, Lx=prob.Lx, Ly=prob.Ly, tau=prob.tau,
          dt=prob.dt)
    for name, a in zip(("w", "w_xi", "w_eta", "X", "Y", "bnd"), arrs):
        setattr(s, name, a.ctypes.data_as(_clib.ctypes.POINTER(ct)))
    return PathInputs(real=real, struct=s, keep=arrs)


def _sfx(inp: PathInputs) -> str:
    return "f32" if inp.real is np.float32 else "f64"


def paths(inp: PathInputs, node_id: int, i0: int, j0: int, p_begin: int, n: int):
    """Per-path records (values (n, 2), steps, exit side, decision margin) of one node."""
    L = _clib.lib()
    val = np.zeros((n, 2), dtype=np.float64)
    steps = np.zeros(n, dtype=np.int32)
    side = np.zeros(n, dtype=np.int8)
    margin = np.zeros(n, dtype=np.float64)
    getattr(L, f"oracle_paths_{_sfx(inp)}")(_clib.ctypes.byref(inp.struct), node_id, i0, j0,
                                            p_begin, n, _clib.ptr(val), _clib.ptr(steps),
                                            _clib.ptr(side), _clib.ptr(margin))
    return val, steps, side, margin


def interface_sums(inp: PathInputs, node_ids, ij, p_begin, n_paths, shift_xy):
    """FP64 shifted sums (S1x, S2x, S1y, S2y) and total substeps per node."""
    L = _clib.lib()
    node_ids = np.ascontiguousarray(node_ids, dtype=np.int32)
    ij = np.ascontiguousarray(ij, dtype=np.int32)
    p_begin = np.ascontiguousarray(p_begin, dtype=np.int64)
    n_paths = np.ascontiguousarray(n_paths, dtype=np.int64)
    shift_xy = np.ascontiguousarray(shift_xy, dtype=np.float64)
    M = len(node_ids)
    sums = np.zeros((M, 4), dtype=np.float64)
    steps = np.zeros(M, dtype=np.int64)
    getattr(L, f"oracle_interface_sums_{_sfx(inp)}")(_clib.ctypes.byref(inp.struct), M,
                                                     _clib.ptr(node_ids), _clib.ptr(ij),
                                                     _clib.ptr(p_begin), _clib.ptr(n_paths),
                                                     _clib.ptr(shift_xy), _clib.ptr(sums),
                                                     _clib.ptr(steps))
    return sums, steps


def estimate(sums, n, shift_xy):
    """Mean, unbiased variance and standard error per node and component from shifted sums.

    mean = s + S1/n,  var = (S2 - S1^2/n) / (n - 1),  SE = sqrt(var / n)  (arithmetic mean
    of Sec. 3.4; the shift s = the node's previous position keeps the sums small).
    """
    sums = np.asarray(sums, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    shift_xy = np.asarray(shift_xy, dtype=np.float64)
    s1 = sums[:, [0, 2]]
    s2 = sums[:, [1, 3]]
    nn = n[:, None]
    mean = shift_xy + s1 / nn
    var = np.maximum((s2 - s1 * s1 / nn) / (nn - 1.0), 0.0)
    se = np.sqrt(var / nn)
    return mean, var, se


def next_total(n_done: int, se: float, target: float, max_paths: int) -> int:
    """Adaptive path count of a node after n_done paths with standard error se.

    Returns n_done when the node is finished (se <= target, or the cap is reached);
    otherwise the new cumulative total: n_done (se/target)^2 times a 1.03 safety factor,
    rounded up to a multiple of 1024 paths, at least 1024 more than n_done, at most max_paths.
    """
    if se <= target or n_done >= max_paths:
        return n_done
    want = n_done * (se / target) ** 2 * ADAPTIVE_SAFETY
    total = int(math.ceil(want / ADAPTIVE_GRANULE)) * ADAPTIVE_GRANULE
    total = max(total, n_done + ADAPTIVE_GRANULE)
    return int(min(total, max_paths))


def interface_mc(prob, x, y, omega, nodes, tstep: int, real=np.float64, bnd=None):
    """Estimates at all interface nodes for one step.

    Fixed N (prob.se_target == 0): paths 0..N-1 of every node.  Adaptive (se_target > 0):
    every node starts with N = prob.paths_per_node paths and draws further chunks, path
    indices continuing, until max(SE_x, SE_y) <= se_target or max_paths_per_node is reached.
    With prob.iface_stride > 1 only the sampled nodes of oracle.layout.interface_sampling are
    estimated (with their own node ids) and the others are interpolated along their lines;
    their se, n_used and steps are 0.
    Returns (est (M,2), se (M,2), n_used (M,), steps (M,)).
    """
    stride = int(getattr(prob, "iface_stride", 0))
    if stride > 1:
        from .layout import interface_sampling
        sampled, fill = interface_sampling(prob.nx, prob.ny, prob.px, prob.py, prob.periodic, stride,
                                           prob.Lx, prob.Ly)
        nodes = np.asarray(nodes, dtype=np.int32)
        sub = _interface_mc_ids(prob, x, y, omega, nodes, np.nonzero(sampled)[0].astype(np.int32), tstep, real, bnd)
        M = len(nodes)
        est = np.full((M, 2), np.nan)
        se = np.zeros((M, 2))
        n_used = np.zeros(M, dtype=np.int64)
        steps = np.zeros(M, dtype=np.int64)
        est[sampled], se[sampled], n_used[sampled], steps[sampled] = sub
        return fill(est), se, n_used, steps
    nodes = np.asarray(nodes, dtype=np.int32)
    return _interface_mc_ids(prob, x, y, omega, nodes, np.arange(len(nodes), dtype=np.int32), tstep, real, bnd)


def _interface_mc_ids(prob, x, y, omega, all_nodes, ids, tstep, real, bnd=None):
    """interface_mc over the nodes all_nodes[ids], each with its own node id in the counter."""
    inp = prepare(prob, x, y, omega, tstep, real, bnd)
    nodes = all_nodes[ids]
    M = len(nodes)
    shift = np.stack([x[nodes[:, 1], nodes[:, 0]], y[nodes[:, 1], nodes[:, 0]]], axis=1)
    n0 = int(prob.paths_per_node)
    sums, steps = interface_sums(inp, ids, nodes, np.zeros(M, np.int64), np.full(M, n0, np.int64),
                                 shift)
    n_used = np.full(M, n0, dtype=np.int64)
    if prob.se_target > 0:
        maxp = int(prob.max_paths_per_node) if prob.max_paths_per_node > 0 else n0
        while True:
            _, _, se = estimate(sums, n_used, shift)
            sem = se.max(axis=1)
            nxt = np.array([next_total(int(n_used[r]), float(sem[r]), prob.se_target, maxp)
                            for r in range(M)], dtype=np.int64)
            todo = np.nonzero(nxt > n_used)[0]
            if len(todo) == 0:
                break
            s2, st2 = interface_sums(inp, ids[todo], nodes[todo], n_used[todo],
                                     nxt[todo] - n_used[todo], shift[todo])
            sums[todo] += s2
            steps[todo] += st2
            n_used[todo] = nxt[todo]
    mean, _, se = estimate(sums, n_used, shift)
    return mean, se, n_used, steps
