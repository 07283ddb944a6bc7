"""Shared helpers of the GPU parity tests: build a problem on both sides from one
workloads.Problem and compare.  The oracle side never takes an input from the CUDA side."""
import numpy as np

import workloads as W
from oracle import mc
from oracle.layout import interface_nodes
from oracle.step import monitor_on_mesh


def real_of(prob):
    return np.float64 if prob.precision == W.PREC_FP64 else np.float32


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


def compare_paths(gpu_val, gpu_steps, gpu_side, or_val, or_steps, or_side, margin, margin_thr, value_tol):
    """Decisions bit-exact and values within value_tol for every path whose decisions all
    clear margin_thr in the oracle; returns (robust fraction, mismatches among the rest)."""
    robust = margin > margin_thr
    assert np.array_equal(gpu_steps[robust], or_steps[robust])
    assert np.array_equal(gpu_side[robust], or_side[robust])
    if robust.any():
        err = np.abs(gpu_val[robust] - or_val[robust]).max()
        assert err <= value_tol, err
    other = ~robust
    mism = int(np.sum((gpu_steps[other] != or_steps[other]) | (gpu_side[other] != or_side[other])))
    return float(robust.mean()), mism
