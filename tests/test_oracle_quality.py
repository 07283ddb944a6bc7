"""Pins of the mesh-quality measure (Eq. 8), the five-ring monitor (Sec. 4.2) and the periodic
single-domain reference solve used for the quality ratio R = Q_SD / Q_SDD (Sec. 3.7)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.layout import interface_nodes
from oracle.monitor import analytic_monitor, monitor_on_grid
from oracle.quality import cell_quality, ratio_stats
from oracle.solve import periodic_single_domain_step
from oracle.step import scatter, subdomain_solves


def grid(nx, ny, Lx=1.0, Ly=1.0):
    xi = np.arange(nx) / (nx - 1)
    eta = np.arange(ny) / (ny - 1)
    X, Y = np.meshgrid(xi, eta)
    return Lx * X, Ly * Y


def test_quality_is_one_on_squares_and_closed_form_on_rectangles():
    x, y = grid(9, 9)
    assert np.allclose(cell_quality(x, y), 1.0, atol=1e-14)
    # cells of aspect ratio a: J = diag(a h, h), Q = (a^2 + 1) / (2 a)
    for a in (2.0, 0.3, 7.5):
        x, y = grid(9, 9, Lx=a, Ly=1.0)
        assert np.allclose(cell_quality(x, y), (a * a + 1) / (2 * a), rtol=1e-13)


def test_quality_at_least_one_and_invariant_under_similarity():
    rng = np.random.default_rng(4)
    x, y = grid(17, 13)
    x = x + 0.01 * rng.normal(size=x.shape)
    y = y + 0.01 * rng.normal(size=y.shape)
    q = cell_quality(x, y)
    assert q.min() >= 1.0 - 1e-12 and q.max() > 1.01
    th, s = 0.7, 3.3
    xr = s * (math.cos(th) * x - math.sin(th) * y) + 5.0
    yr = s * (math.sin(th) * x + math.cos(th) * y) - 2.0
    assert np.allclose(cell_quality(xr, yr), q, rtol=1e-12)


def test_quality_of_a_sheared_cell():
    # unit square sheared by s: x_xi = (1, 0), x_eta = (s, 1): Q = (2 + s^2) / 2
    s = 0.4
    x = np.array([[0.0, 1.0], [s, 1.0 + s]])
    y = np.array([[0.0, 0.0], [1.0, 1.0]])
    assert abs(cell_quality(x, y)[0, 0] - (2 + s * s) / 2) < 1e-14


def test_ratio_stats():
    a = np.array([[1.0, 2.0], [1.5, 1.0]])
    b = np.array([[1.0, 1.0], [1.5, 2.0]])
    r = ratio_stats(a, b)
    assert r["R_max"] == 2.0 and r["R_mean"] == (1 + 2 + 1 + 0.5) / 4 and r["maxQ_ratio"] == 1.0


def test_ring_monitor_gradient_matches_numerical_derivative():
    prob = W.five_ring(2)
    alpha, R, r2 = prob.monitor_params[:3]
    cs = prob.monitor_params[3:]
    rng = np.random.default_rng(1)
    x = rng.uniform(0.2, 1.8, 300)
    y = rng.uniform(0.2, 1.8, 300)
    u = lambda a, b: sum(np.tanh(R * ((a - cs[k]) ** 2 + (b - cs[k + 1]) ** 2 - r2)) for k in range(0, 10, 2))
    h = 1e-6
    gx = (u(x + h, y) - u(x - h, y)) / (2 * h)
    gy = (u(x, y + h) - u(x, y - h)) / (2 * h)
    got = analytic_monitor(W.MONITOR_RINGS, prob.monitor_params, x, y, 0.0)
    assert np.allclose(got, np.sqrt(1 + alpha * (gx ** 2 + gy ** 2)), rtol=1e-6)


def test_periodic_single_domain_keeps_uniform_mesh_and_decays_mode():
    nx = 17
    Lx, Ly = 2.0, 1.5
    x, y = grid(nx, nx, Lx, Ly)
    om = np.full((nx, nx), 2.0)
    x1, y1 = periodic_single_domain_step(om, x, y, 1e-3, 1e-2, 0, Lx, Ly)
    assert np.allclose(x1, x, atol=1e-13) and np.allclose(y1, y, atol=1e-13)
    # periodic Fourier mode: factor 1 / (1 + r c mu), mu = sum over directions (4/h^2) sin^2(pi h)
    A = 0.01
    xi, eta = grid(nx, nx)
    mode = np.sin(2 * np.pi * xi) * np.sin(2 * np.pi * eta)
    x1, y1 = periodic_single_domain_step(om, x + A * mode, y + A * mode, 1e-3, 1e-2, 0, Lx, Ly)
    h = 1.0 / (nx - 1)
    mu = 2 * (4 / h ** 2) * math.sin(math.pi * h) ** 2
    fac = 1 / (1 + 0.1 * 2.0 * mu)
    assert np.allclose(x1, x + A * fac * mode, atol=1e-13)
    assert np.allclose(y1, y + A * fac * mode, atol=1e-13)


@pytest.mark.parametrize("px", [2, 4])
def test_periodic_subdomains_with_exact_interface_data_reproduce_single_domain(px):
    prob = W.five_ring(px).replace(nx=33, ny=33)
    x, y = grid(33, 33, prob.Lx, prob.Ly)
    x = x + 0.01 * np.sin(2 * np.pi * x / 2) * np.sin(2 * np.pi * y / 2)
    om = monitor_on_grid(prob.monitor_kind, prob.monitor_params, x, y, 0.0, 1, prob.Lx, prob.Ly)
    xs, ys = periodic_single_domain_step(om, x, y, prob.dt, prob.tau, prob.form, prob.Lx, prob.Ly)
    nodes = interface_nodes(33, 33, px, px, 1)
    est = np.stack([xs[nodes[:, 1], nodes[:, 0]], ys[nodes[:, 1], nodes[:, 0]]], 1)
    bx, by = scatter(prob, nodes, est)
    x1, y1 = subdomain_solves(prob, om, bx, by, x, y)
    assert np.allclose(x1, xs, atol=1e-12) and np.allclose(y1, ys, atol=1e-12)


def test_five_ring_single_substep_estimate_is_the_explicit_drift_step():
    """Why the paper's one-substep setting (Sec. 4.2, ds = dt) does not keep the single-domain
    mesh quality at 41 x 41 nodes.  On the uniform initial mesh (x linear in xi, so the previous
    mesh is interpolated exactly) the expectation of x0(Phi^1) is x0 at the end of the drift step,
    xi + (grad omega / omega) dt: the estimates equal that explicit step within 4.5 standard errors
    at every interface node.  At the rings this step moves nodes by up to 1.5 cells and
    dt |d b / d xi| exceeds 1, so the estimates overshoot the backward-Euler single-domain solution
    by more than half a cell; with 16 substeps they stay within a fifth of a cell of it."""
    from oracle import step as ostep
    from oracle.monitor import fd_gradient
    prob = W.five_ring(2)
    x, y = grid(prob.nx, prob.ny, prob.Lx, prob.Ly)
    om = monitor_on_grid(prob.monitor_kind, prob.monitor_params, x, y, 0.0, 1, prob.Lx, prob.Ly)
    gx, gy = fd_gradient(om, 1)
    bx, by = gx / om, gy / om        # drift of the paper's generator (tau = 1)
    h = 1.0 / (prob.nx - 1)
    db = max(np.abs((np.roll(bx, -1, 1) - np.roll(bx, 1, 1)) / (2 * h)).max(),
             np.abs((np.roll(by, -1, 0) - np.roll(by, 1, 0)) / (2 * h)).max())
    assert prob.dt * db > 1.0
    assert max(np.abs(bx).max(), np.abs(by).max()) * prob.dt / h > 1.4
    r = ostep.step(prob, x, y, 0.0, 0)
    ii, jj = r["nodes"][:, 0], r["nodes"][:, 1]
    expl = np.stack([x[jj, ii] + prob.Lx * bx[jj, ii] * prob.dt, y[jj, ii] + prob.Ly * by[jj, ii] * prob.dt], 1)
    assert np.all(np.abs(r["est"] - expl) <= 4.5 * r["se"] + 1e-12)
    xs, ys = periodic_single_domain_step(om, x, y, prob.dt, prob.tau, prob.form, prob.Lx, prob.Ly)
    sd = np.stack([xs[jj, ii], ys[jj, ii]], 1)
    cell = prob.Lx * h
    assert np.abs(r["est"] - sd).max() > 0.5 * cell
    r16 = ostep.step(prob.replace(substeps=16), x, y, 0.0, 0)
    assert np.abs(r16["est"] - sd).max() < 0.2 * cell
