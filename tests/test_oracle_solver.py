"""Pins of the oracle's backward-Euler subdomain / single-domain solves (Sec. 3.5, 3.6)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.layout import interface_nodes
from oracle.solve import box_system, single_domain_step, solve_box
from oracle.step import scatter, subdomain_solves


def grid(nx, ny):
    xi = np.arange(nx) / (nx - 1)
    eta = np.arange(ny) / (ny - 1)
    return np.meshgrid(xi, eta)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("nx,ny", [(17, 17), (33, 17)])
def test_discrete_sine_mode_is_an_eigenvector(form, nx, ny):
    """Constant omega = c on a uniform grid: the discrete mode sin(pi xi) sin(pi eta) is an
    eigenvector of the 5-point operator with eigenvalue
    mu = (4/h_xi^2) sin^2(pi h_xi/2) + (4/h_eta^2) sin^2(pi h_eta/2), so one backward-Euler step
    multiplies it by 1 / (1 + r c mu) (form 0) or 1 / (1 + r mu) (form 1)."""
    c, dt, tau, A = 2.5, 1e-3, 1e-2, 0.05
    XI, ETA = grid(nx, ny)
    mode = np.sin(np.pi * XI) * np.sin(np.pi * ETA)
    om = np.full((ny, nx), c)
    x0, y0 = XI + A * mode, ETA + A * mode
    x1, y1 = single_domain_step(om, x0, y0, dt, tau, form)
    hx, hy = 1 / (nx - 1), 1 / (ny - 1)
    mu = 4 / hx ** 2 * math.sin(math.pi * hx / 2) ** 2 + 4 / hy ** 2 * math.sin(math.pi * hy / 2) ** 2
    r = dt / tau
    fac = 1 / (1 + r * c * mu) if form == 0 else 1 / (1 + r * mu)
    assert np.allclose(x1, XI + A * fac * mode, atol=1e-13)
    assert np.allclose(y1, ETA + A * fac * mode, atol=1e-13)


@pytest.mark.parametrize("form", [0, 1])
def test_discrete_equidistribution_is_steady(form):
    """omega = omega(xi): the mesh whose face fluxes (omega_i + omega_{i+1})/2 (x_{i+1} - x_i)
    are all equal, with y = eta, is a fixed point of the step (variable coefficients)."""
    nx, ny = 21, 13
    xi = np.arange(nx) / (nx - 1)
    w = np.exp(1.7 * xi) + 0.3 * np.sin(5 * xi)
    wf = 0.5 * (w[1:] + w[:-1])
    xs = np.concatenate([[0.0], np.cumsum(1.0 / wf)])
    xs /= xs[-1]
    x0 = np.tile(xs, (ny, 1))
    _, y0 = grid(nx, ny)
    om = np.tile(w, (ny, 1))
    xs1, ys1, order = solve_box(om, x0, y0, x0, y0, 0, nx - 1, 0, ny - 1, 5e-3, 1e-3, form)
    for P, (i, j) in enumerate(order):
        assert abs(xs1[P] - x0[j, i]) < 1e-12 and abs(ys1[P] - y0[j, i]) < 1e-12
    # adding an eta-dependent term to the monitor changes the face fluxes: no longer steady
    om2 = om + 0.5 * np.tile(np.arange(ny)[:, None] / (ny - 1), (1, nx))
    xs2, _, _ = solve_box(om2, x0, y0, x0, y0, 0, nx - 1, 0, ny - 1, 5e-3, 1e-3, form)
    assert max(abs(xs2[P] - x0[j, i]) for P, (i, j) in enumerate(order)) > 1e-4


@pytest.mark.parametrize("form", [0, 1])
def test_solution_minimises_the_discrete_energy(form):
    """Brute force on a tiny box: the solve minimises
    E(x) = 1/2 sum_P d_P (x_P - x^n_P)^2 + r/2 sum_faces w_f (x_a - x_b)^2 / h_f^2
    (d_P = 1 for form 0, omega_P for form 1) over the interior values, rim held fixed."""
    rng = np.random.default_rng(0)
    nx, ny = 6, 5
    om = rng.uniform(0.5, 3.0, size=(ny, nx))
    xn = rng.normal(size=(ny, nx))
    rim = rng.normal(size=(ny, nx))
    dt, tau = 0.3, 1.0
    r = dt / tau
    xs, _, order = solve_box(om, rim, rim, xn, xn, 0, nx - 1, 0, ny - 1, dt, tau, form)
    inner = set(order)

    def energy(vals):
        f = rim.copy()
        for P, (i, j) in enumerate(order):
            f[j, i] = vals[P]
        e = 0.0
        for (i, j) in order:
            d = 1.0 if form == 0 else om[j, i]
            e += 0.5 * d * (f[j, i] - xn[j, i]) ** 2
        for j in range(ny):
            for i in range(nx):
                for (a, b, h2) in (((i + 1, j), (i, j), (nx - 1) ** 2), ((i, j + 1), (i, j), (ny - 1) ** 2)):
                    if a[0] >= nx or a[1] >= ny:
                        continue
                    if a not in inner and b not in inner:
                        continue
                    wf = 0.5 * (om[a[1], a[0]] + om[b[1], b[0]])
                    e += 0.5 * r * wf * h2 * (f[a[1], a[0]] - f[b[1], b[0]]) ** 2
        return e

    e0 = energy(xs)
    n = len(xs)
    eps = 1e-4
    for k in range(n):
        v = np.zeros(n); v[k] = eps
        g = (energy(xs + v) - energy(xs - v)) / (2 * eps)
        assert abs(g) < 1e-6 * max(1.0, abs(e0))
    for _ in range(20):
        v = rng.normal(size=n) * 1e-3
        assert energy(xs + v) > e0


def test_matrix_is_symmetric_positive_definite():
    rng = np.random.default_rng(1)
    om = rng.uniform(1.0, 5.0, size=(9, 11))
    for form in (0, 1):
        A, _, _ = box_system(om, None, 0, 10, 0, 8, 0.01, 0.1, form)
        Ad = A.toarray()
        assert np.allclose(Ad, Ad.T)
        lam = np.linalg.eigvalsh(Ad)
        assert lam.min() >= (1.0 if form == 0 else om.min()) - 1e-9


@pytest.mark.parametrize("px,py", [(2, 2), (4, 2)])
def test_subdomains_with_exact_interface_data_reproduce_single_domain(px, py):
    """Fed the single-domain solution on the interfaces, the independent subdomain solves
    return the single-domain solution (the subdomain equations are rows of the global system)."""
    prob = W.Problem(name="t", nx=33, ny=17, px=px, py=py, dt=2e-3, tau=1e-2)
    XI, ETA = grid(prob.nx, prob.ny)
    om = 1 + 4 * np.exp(-30 * ((XI - 0.4) ** 2 + (ETA - 0.6) ** 2))
    x0 = XI + 0.03 * np.sin(np.pi * XI) * np.sin(2 * np.pi * ETA)
    y0 = ETA + 0.02 * np.sin(3 * np.pi * XI) * np.sin(np.pi * ETA)
    xs, ys = single_domain_step(om, x0, y0, prob.dt, prob.tau, 0)
    nodes = interface_nodes(prob.nx, prob.ny, px, py)
    est = np.stack([xs[nodes[:, 1], nodes[:, 0]], ys[nodes[:, 1], nodes[:, 0]]], 1)
    bx, by = scatter(prob, nodes, est)
    x1, y1 = subdomain_solves(prob, om, bx, by, x0, y0)
    assert np.allclose(x1, xs, atol=1e-12) and np.allclose(y1, ys, atol=1e-12)


def test_periodic_scatter_applies_period_offsets():
    prob = W.Problem(name="t", nx=9, ny=9, px=2, py=2, periodic=1, Lx=2.0, Ly=3.0)
    nodes = interface_nodes(9, 9, 2, 2, 1)
    est = np.stack([2.0 * nodes[:, 0] / 8, 3.0 * nodes[:, 1] / 8], 1)
    bx, by = scatter(prob, nodes, est)
    assert np.allclose(bx[:, 8][~np.isnan(bx[:, 8])], 2.0)
    assert bx[0, 8] == 2.0 and by[8, 0] == 3.0 and bx[8, 8] == 2.0 and by[8, 8] == 3.0
    # all rims of all subdomains are defined
    for (i0, i1, j0, j1) in [(0, 4, 0, 4), (4, 8, 0, 4), (0, 4, 4, 8), (4, 8, 4, 8)]:
        for i in range(i0, i1 + 1):
            for j in (j0, j1):
                assert not np.isnan(bx[j, i]) and not np.isnan(by[j, i])
        for j in range(j0, j1 + 1):
            for i in (i0, i1):
                assert not np.isnan(bx[j, i])


def test_forward_euler_periodic_mode_decay_closed_form():
    """Constant omega on the periodic grid: the mode sin(2 pi xi) sin(2 pi eta) is an eigenvector of
    the operator with eigenvalue r w mu, mu = 2 (4/h^2) sin^2(pi h); each of the S substeps
    multiplies it by 1 - r w mu / S, S = ceil(4 r w / h^2) (the largest sum of coefficients)."""
    import math
    from oracle.solve import periodic_single_domain_step_fe
    nx = 17
    Lx, Ly = 2.0, 1.5
    xi = np.arange(nx) / (nx - 1)
    X, Y = np.meshgrid(xi, xi)
    w0, dt, tau = 2.0, 1e-3, 1e-2
    om = np.full((nx, nx), w0)
    x1, y1 = periodic_single_domain_step_fe(om, Lx * X, Ly * Y, dt, tau, 0, Lx, Ly)
    assert np.allclose(x1, Lx * X, atol=1e-13) and np.allclose(y1, Ly * Y, atol=1e-13)
    A = 0.01
    mode = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    x1, y1 = periodic_single_domain_step_fe(om, Lx * X + A * mode, Ly * Y + A * mode, dt, tau, 0, Lx, Ly)
    h = 1.0 / (nx - 1)
    r = dt / tau
    S = math.ceil(4 * r * w0 / h ** 2)
    lam = r * w0 * 2 * (4 / h ** 2) * math.sin(math.pi * h) ** 2
    fac = (1 - lam / S) ** S
    assert np.allclose(x1, Lx * X + A * fac * mode, atol=1e-13)
    assert np.allclose(y1, Ly * Y + A * fac * mode, atol=1e-13)


def test_forward_euler_box_keeps_linear_meshes_and_counts_substeps():
    from oracle.solve import solve_box_fe
    nx = 17
    xi = np.arange(nx) / (nx - 1)
    X, Y = np.meshgrid(xi, xi)
    om = np.full((nx, nx), 3.0)
    xs, ys, order, S = solve_box_fe(om, X, Y, X, Y, 0, 8, 4, 16, 1e-3, 1e-2, 0)
    want = np.array([X[j, i] for i, j in order]), np.array([Y[j, i] for i, j in order])
    assert np.allclose(xs, want[0], atol=1e-14) and np.allclose(ys, want[1], atol=1e-14)
    assert S == int(np.ceil(4 * 0.1 * 3.0 * 256 - 1e-9))


def test_forward_euler_agrees_with_backward_euler_to_second_order():
    """Both are first-order steps of the same linear ODE: FE - BE = O(r^2) on a smooth mesh."""
    from oracle.solve import solve_box, solve_box_fe
    nx = 17
    xi = np.arange(nx) / (nx - 1)
    X, Y = np.meshgrid(xi, xi)
    om = 1.0 + 0.5 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    xm = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    errs = []
    for dt in (1e-4, 5e-5):
        fx, _, order, _ = solve_box_fe(om, X, Y, xm, Y, 0, 16, 0, 16, dt, 1.0, 0)
        bx, _, _ = solve_box(om, X, Y, xm, Y, 0, 16, 0, 16, dt, 1.0, 0)
        errs.append(np.abs(fx - bx).max())
    assert errs[1] < errs[0] / 3.0   # second order in dt: halving dt quarters the gap
