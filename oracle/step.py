"""One alternating time step of the SDD mesh generator -- oracle, TEST INFRASTRUCTURE.

The domain decomposition solution (Sec. 3.6): with the monitor frozen on the current mesh
(Sec. 3.2), the interface nodes are estimated stochastically (Sec. 3.4), the estimates are
the Dirichlet data of independent subdomain solves (Sec. 3.5), and the new mesh is the union
of interface values, subdomain interiors and the physical boundary.
"""
from __future__ import annotations

import numpy as np

from workloads import MONITOR_NODAL
from .layout import interface_nodes, subdomains
from .mc import interface_mc
from .monitor import monitor_on_grid, wrap_copy
from .solve import solve_box, solve_box_fe


def monitor_on_mesh(prob, x, y, t, omega_nodal=None):
    if prob.monitor_kind == MONITOR_NODAL:
        if omega_nodal is None:
            raise ValueError("nodal monitor needs omega")
        om = np.asarray(omega_nodal, dtype=np.float64)
        return wrap_copy(om) if prob.periodic else om
    return monitor_on_grid(prob.monitor_kind, prob.monitor_params, x, y, t, prob.periodic,
                            prob.Lx, prob.Ly)


def scatter(prob, nodes, est, bnd=None):
    """New-mesh arrays holding the Dirichlet data of every subdomain rim.

    Dirichlet: the physical boundary keeps the identity mesh (Lx xi, Ly eta); interface
    nodes take the estimates.  Periodic: interface nodes take the estimates and the wrap
    column/row carries the period offset, x(1, eta) = x(0, eta) + Lx, y(xi, 1) = y(xi, 0) + Ly.
    Nodes that are neither are left as NaN (they are subdomain interiors).
    """
    nx, ny = prob.nx, prob.ny
    bx = np.full((ny, nx), np.nan)
    by = np.full((ny, nx), np.nan)
    if bnd is not None:           # moving boundary: the new boundary mesh (oracle.boundary)
        from .boundary import boundary_arrays
        bx, by = boundary_arrays(prob, bnd)
    elif not prob.periodic:
        xi = np.arange(nx) / (nx - 1)
        eta = np.arange(ny) / (ny - 1)
        bx[0, :] = prob.Lx * xi; bx[-1, :] = prob.Lx * xi
        by[0, :] = 0.0; by[-1, :] = prob.Ly
        bx[:, 0] = 0.0; bx[:, -1] = prob.Lx
        by[:, 0] = prob.Ly * eta; by[:, -1] = prob.Ly * eta
    for (i, j), (vx, vy) in zip(nodes, est):
        bx[j, i] = vx
        by[j, i] = vy
        if prob.periodic:
            if i == 0:
                bx[j, nx - 1] = vx + prob.Lx; by[j, nx - 1] = vy
            if j == 0:
                bx[ny - 1, i] = vx; by[ny - 1, i] = vy + prob.Ly
            if i == 0 and j == 0:
                bx[ny - 1, nx - 1] = vx + prob.Lx; by[ny - 1, nx - 1] = vy + prob.Ly
    return bx, by


def subdomain_solves(prob, omega, bx, by, xn, yn):
    """Fill every subdomain interior of (bx, by) by its backward-Euler solve (Sec. 3.5), or by
    forward-Euler substeps when prob.subdomain_scheme == 1 (the paper's local solver)."""
    out_x, out_y = bx.copy(), by.copy()
    fe = int(getattr(prob, "subdomain_scheme", 0)) == 1
    for (i0, i1, j0, j1) in subdomains(prob.nx, prob.ny, prob.px, prob.py):
        if fe:
            xs, ys, order, _ = solve_box_fe(omega, bx, by, xn, yn, i0, i1, j0, j1, prob.dt, prob.tau,
                                            prob.form)
        else:
            xs, ys, order = solve_box(omega, bx, by, xn, yn, i0, i1, j0, j1, prob.dt, prob.tau,
                                      prob.form)
        for P, (i, j) in enumerate(order):
            out_x[j, i] = xs[P]
            out_y[j, i] = ys[P]
    return out_x, out_y


def step(prob, x, y, t, tstep, omega_nodal=None, real=np.float64):
    """x^n -> x^{n+1}.  Returns dict with the new mesh, interface estimates, SE, paths, steps."""
    omega = monitor_on_mesh(prob, x, y, t, omega_nodal)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic)
    bnd = None
    if int(getattr(prob, "moving_boundary", 0)):
        from .boundary import boundary_mesh_step
        bnd = boundary_mesh_step(prob, omega, x, y)   # the boundary first (Sec. 2), then the interfaces
    est, se, n_used, steps = interface_mc(prob, x, y, omega, nodes, tstep, real, bnd)
    bx, by = scatter(prob, nodes, est, bnd)
    xn1, yn1 = subdomain_solves(prob, omega, bx, by, x, y)
    return dict(x=xn1, y=yn1, est=est, se=se, n_used=n_used, steps=steps, omega=omega,
                nodes=nodes, bnd=bnd)


def mkp_step(prob, x, y, t, tstep, K, omega_nodal=None, real=np.float64):
    """M^kP step (Sec. 5): x^n -> x^{n+1} through K sub-meshes, each a step of dt/K with the
    monitor evaluated on the current sub-mesh at the step's time t (the analytic monitor at the
    sub-mesh positions in place of the paper's interpolant of rho^n); sub-step k uses the
    counter word tstep K + k.  Returns the last sub-step's dict (new mesh in x, y)."""
    sub = prob.replace(dt=prob.dt / K)
    r = None
    for k in range(K):
        r = step(sub, x, y, t, tstep * K + k, omega_nodal, real)
        x, y = r["x"], r["y"]
    return r
