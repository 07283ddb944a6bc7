"""Shared helpers of the GPU parity tests: build a problem on both sides from one
workloads.Problem and compare.  The oracle side never takes an input from the CUDA side."""
import numpy as np

import workloads as W
from oracle import mc
from oracle.layout import interface_nodes
from oracle.step import monitor_on_mesh

# Per-path tolerances: values within 1e-12 (FP64) or 1e-5 (FP32) of the oracle's.  Exit step and
# side are compared bit for bit on every path; a decision may differ only where the oracle's
# decision margin (distance of the deciding quantity from its threshold) is at most about one
# rounding unit of the working precision: 1e-12 (FP64) or 1e-7 (FP32, about two units in the
# last place at 1).  Such near-tie paths may be at most NEAR_TIE_MAX of all compared paths.
FP64_MARGIN, FP64_VAL = 1e-12, 1e-12
FP32_MARGIN, FP32_VAL = 1e-7, 1e-5
NEAR_TIE_MAX = 1e-3


def real_of(prob):
    return np.float64 if prob.precision == W.PREC_FP64 else np.float32


def tolerances(prob):
    """(margin threshold, value tolerance) of the problem's path precision."""
    if prob.precision == W.PREC_FP64:
        return FP64_MARGIN, FP64_VAL
    return FP32_MARGIN, FP32_VAL


def gpu_problem(prob, x=None, y=None, omega=None):
    import paper_1504_00084_gb300 as S
    if x is None:
        x, y = W.identity_mesh(prob)
    h = S.SddProblem(S.params_from(prob), x, y)
    if prob.monitor_kind == W.MONITOR_NODAL:
        if omega is not None:
            h.set_monitor(omega)
    else:
        h.set_monitor_analytic(prob.monitor_kind, prob.monitor_params)
    return h


def oracle_inputs(prob, x, y, t, tstep, omega=None):
    om = monitor_on_mesh(prob, x, y, t, omega)
    bnd = None
    if getattr(prob, "moving_boundary", 0):
        from oracle.boundary import boundary_mesh_step
        bnd = boundary_mesh_step(prob, om, x, y)
    inp = mc.prepare(prob, x, y, om, tstep, real_of(prob), bnd)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic)
    return om, inp, nodes


class PathTally:
    """Running totals of per-path comparisons over several nodes."""

    def __init__(self):
        self.n = 0
        self.near = 0
        self.mism = 0
        self.agree = 0
        self.within = 0
        self.max_err = 0.0

    def add(self, gpu_val, gpu_steps, gpu_side, or_val, or_steps, or_side, margin, margin_thr, value_tol):
        """Add one node's paths.  Asserts at once that every path whose oracle margin clears
        margin_thr has the oracle's exit step and side; counts the near-tie paths, the decision
        mismatches among them, and the paths with agreeing decisions whose values are within
        value_tol."""
        near = margin <= margin_thr
        same = (gpu_steps == or_steps) & (gpu_side == or_side)
        assert same[~near].all(), "exit decision differs on a path with a clear margin"
        err = np.abs(gpu_val - or_val).max(axis=1)[same]
        self.n += len(margin)
        self.near += int(near.sum())
        self.mism += int((~same).sum())
        self.agree += int(same.sum())
        self.within += int((err <= value_tol).sum())
        if len(err):
            self.max_err = max(self.max_err, float(err.max()))
        return self

    def check(self, value_frac=1.0, max_near=NEAR_TIE_MAX):
        """Near-tie paths at most max_near of all; values within tolerance on every path whose
        decisions agree (value_frac = 1), or on at least that fraction of them."""
        assert self.n > 0
        assert self.near <= max_near * self.n, (self.near, self.n)
        assert self.mism <= self.near
        if value_frac >= 1.0:
            assert self.within == self.agree, (self.agree - self.within, self.max_err)
        else:
            assert self.within >= value_frac * self.agree, (self.within, self.agree, self.max_err)
        return self


def compare_node_paths(h, inp, nodes, node_ids, n, prob, tally=None):
    """Per-path records of n paths at each node of node_ids, GPU (debug hook of the production
    kernel body) against the oracle, added to a PathTally."""
    margin_thr, value_tol = tolerances(prob)
    tally = tally or PathTally()
    for m in node_ids:
        gv, gs, gd = h.debug_paths(int(m), 0, n)
        ov, os_, od, mg = mc.paths(inp, int(m), int(nodes[m, 0]), int(nodes[m, 1]), 0, n)
        tally.add(gv, gs, gd, ov, os_, od, mg, margin_thr, value_tol)
    return tally


def mesh_tolerance(prob, om, rims_x, rims_y, xn, yn, est_tol):
    """Interface tolerance (the discrete maximum principle carries it into the interiors) plus the
    solver's bound ||x - x*||_2 <= ||A^-1|| rtol ||b||_2 with ||A^-1|| <= 1 / lambda_min,
    lambda_min >= 1 (form 0) or >= min omega (form 1)."""
    from oracle.layout import subdomains
    from oracle.solve import box_system
    lam = 1.0 if prob.form == W.FORM_DIV else float(om.min())
    worst = 0.0
    for (i0, i1, j0, j1) in subdomains(prob.nx, prob.ny, prob.px, prob.py):
        if i1 - i0 < 2 or j1 - j0 < 2:
            continue
        A, rhs, _ = box_system(om, None, i0, i1, j0, j1, prob.dt, prob.tau, prob.form)
        bx = np.linalg.norm(rhs(rims_x, xn))
        by = np.linalg.norm(rhs(rims_y, yn))
        worst = max(worst, prob.solve_rtol * max(bx, by) / lam)
    return est_tol + worst + 1e-12
