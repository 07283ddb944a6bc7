"""Pins of the oracle's path simulator and estimator against closed forms of the stochastic
representation (Eq. 5a, 5b, 6, 7) and against the exit-time laws of Brownian motion."""
import math

import numpy as np
import pytest
import scipy.special

import workloads as W
from oracle import mc
from oracle.monitor import wrap_copy


def Phi(z):
    return 0.5 * scipy.special.erfc(-z / math.sqrt(2.0))


def make(nx=65, periodic=0, form=W.FORM_DIV, tau=1.0, dt=1e-3, K=1, bb=1, bicubic=1, seed=11):
    return W.Problem(name="t", nx=nx, ny=nx, px=2, py=2, periodic=periodic, form=form, tau=tau,
                     dt=dt, substeps=K, bb_test=bb, bicubic=bicubic, seed=seed,
                     monitor_kind=W.MONITOR_NODAL)


def prepared(prob, omega, x=None, y=None, real=np.float64, tstep=0):
    if x is None:
        x, y = W.identity_mesh(prob)
    return mc.prepare(prob, x, y, omega, tstep, real)


def node_mean(inp, i0, j0, n, shift=(0.0, 0.0), node_id=0):
    sums, steps = mc.interface_sums(inp, [node_id], [[i0, j0]], [0], [n], [shift])
    mean, var, se = mc.estimate(sums, np.array([n]), np.array([shift]))
    return mean[0], se[0], steps[0]


# ---------------------------------------------------------------------------------------
# Exit laws of Brownian motion (constant omega: no drift, D = omega / tau or 1 / tau).
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("bb", [1, 0])
@pytest.mark.parametrize("form,omega_c", [(W.FORM_DIV, 2.0), (W.FORM_WINSLOW, 2.0)])
def test_single_substep_exit_probability(oracle_lib, bb, form, omega_c):
    """One substep from distance d of the side xi = 0.  With the bridge test the exit
    probability is the reflection-principle value 2 Phi(-d / sqrt(2 D ds)); without it only
    the endpoint counts, Phi(-d / sqrt(2 D ds))."""
    prob = make(form=form, bb=bb, K=1, dt=1e-3, tau=1.0)
    om = np.full((prob.ny, prob.nx), omega_c)
    inp = prepared(prob, om)
    i0, j0 = 2, 32
    d = i0 / (prob.nx - 1)
    D = omega_c / prob.tau if form == W.FORM_DIV else 1.0 / prob.tau
    s = math.sqrt(2 * D * prob.dt)
    n = 200000
    val, steps, side, _ = mc.paths(inp, 0, i0, j0, 0, n)
    frac = np.mean(side == 0)
    expect = (2.0 if bb else 1.0) * Phi(-d / s)
    assert abs(frac - expect) < 4 * math.sqrt(expect * (1 - expect) / n) + 1e-4
    assert np.all(side[side != 0] == 4)
    assert np.all(val[side == 0, 0] == 0.0)


def strip_survival(x0, DT, terms=200):
    """P(1-D Brownian motion with diffusion D started at x0 stays in (0, 1) up to T)."""
    k = np.arange(1, 2 * terms, 2)
    return float(np.sum(4.0 / (k * np.pi) * np.sin(k * np.pi * x0) * np.exp(-(k * np.pi) ** 2 * DT)))


@pytest.mark.parametrize("form", [W.FORM_DIV, W.FORM_WINSLOW])
def test_survival_in_the_square_matches_heat_kernel_series(oracle_lib, form):
    """K substeps with the bridge test: survival in the unit square equals the product of the
    two 1-D strip survival series (independent components)."""
    omega_c = 1.5
    prob = make(form=form, K=100, dt=0.05, tau=1.0, bb=1)
    om = np.full((prob.ny, prob.nx), omega_c)
    inp = prepared(prob, om)
    D = omega_c / prob.tau if form == W.FORM_DIV else 1.0 / prob.tau
    for (i0, j0) in [(32, 32), (16, 40)]:
        n = 100000
        _, steps, side, _ = mc.paths(inp, 0, i0, j0, 0, n)
        frac = np.mean(side == 4)
        expect = strip_survival(i0 / 64, D * prob.dt) * strip_survival(j0 / 64, D * prob.dt)
        assert abs(frac - expect) < 4 * math.sqrt(expect * (1 - expect) / n) + 2e-3, (frac, expect)
        assert np.all(steps[side == 4] == prob.substeps)
        assert np.all((steps[side != 4] >= 1) & (steps[side != 4] <= prob.substeps))


# ---------------------------------------------------------------------------------------
# Closed-form solutions of the linear generator.
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("real", [np.float64, np.float32])
def test_uniform_mesh_stays_uniform(oracle_lib, periodic, real):
    """Constant omega, identity mesh: every path value is a martingale with unbiased exit
    values, so E[x] = Lx xi at each node."""
    prob = make(periodic=periodic, K=50, dt=0.02, tau=1.0, seed=5)
    prob = prob.replace(Lx=2.0, Ly=0.5)
    om = np.full((prob.ny, prob.nx), 3.0)
    inp = prepared(prob, om, real=real)
    for (i0, j0) in [(16, 16), (32, 48), (5, 60)]:
        n = 50000
        pos = (prob.Lx * i0 / 64, prob.Ly * j0 / 64)
        mean, se, _ = node_mean(inp, i0, j0, n, shift=pos)
        assert np.all(np.abs(mean - pos) < 4 * se + 1e-6), (mean, pos, se)


def test_sine_mode_decays_as_closed_form_dirichlet(oracle_lib):
    """omega = 1, x0 = xi + A sin(pi xi) sin(pi eta): x(t) = xi + A exp(-2 pi^2 t / tau) sin sin."""
    prob = make(K=100, dt=0.01, tau=1.0, seed=3)
    om = np.ones((prob.ny, prob.nx))
    A = 0.05
    x0, y0 = W.sine_mode_mesh(prob, amp=A)
    inp = prepared(prob, om, x0, y0)
    fac = math.exp(-2 * math.pi ** 2 * prob.dt / prob.tau)
    wrong = math.exp(-math.pi ** 2 * prob.dt / prob.tau)   # what a halved diffusion would give
    for (i0, j0) in [(32, 32), (20, 40)]:
        xi, eta = i0 / 64, j0 / 64
        mode = A * math.sin(math.pi * xi) * math.sin(math.pi * eta)
        n = 100000
        mean, se, _ = node_mean(inp, i0, j0, n, shift=(xi, eta))
        expect = np.array([xi, eta]) + mode * fac
        assert np.all(np.abs(mean - expect) < 4 * se + 1e-5), (mean, expect, se)
        assert np.all(np.abs(mean - (np.array([xi, eta]) + mode * wrong)) > 4 * se)


def test_sine_mode_decays_as_closed_form_periodic(oracle_lib):
    """Periodic: x0 = xi + A sin(2 pi xi) sin(2 pi eta) decays by exp(-8 pi^2 t / tau) (Eq. 6)."""
    prob = make(periodic=1, K=50, dt=0.01, tau=1.0, seed=9)
    om = np.ones((prob.ny, prob.nx))
    A = 0.05
    x0, y0 = W.sine_mode_mesh(prob, amp=A, periodic_mode=True)
    inp = prepared(prob, om, x0, y0)
    fac = math.exp(-8 * math.pi ** 2 * prob.dt / prob.tau)
    for (i0, j0) in [(16, 16), (0, 16), (48, 8)]:
        xi, eta = i0 / 64, j0 / 64
        mode = A * math.sin(2 * math.pi * xi) * math.sin(2 * math.pi * eta)
        n = 100000
        mean, se, _ = node_mean(inp, i0, j0, n, shift=(xi, eta))
        expect = np.array([xi, eta]) + mode * fac
        assert np.all(np.abs(mean - expect) < 4 * se + 1e-5), (mean, expect, se)


@pytest.mark.parametrize("form", [W.FORM_DIV, W.FORM_WINSLOW])
def test_steady_state_with_variable_monitor_needs_the_drift(oracle_lib, form):
    """omega = exp(c xi): x = (1 - exp(-c xi)) / (1 - exp(-c)), y = eta is a steady state of both
    generator forms, so the estimate must return the node's own position.  Without the drift
    term (or with its sign flipped) the estimate moves by O(dt omega x'' / tau) >> SE.
    Nodes sit on eta = 1/2, about five diffusion lengths from the sides eta = 0, 1 where the
    fixed identity boundary differs from this steady state; on the sides xi = 0, 1 the two agree."""
    c = 2.0
    dt = 2e-3 if form == W.FORM_DIV else 5e-3   # both about five diffusion lengths from eta = 0, 1
    prob = make(nx=65, form=form, K=100, dt=dt, tau=1.0, seed=21)
    xi = np.arange(prob.nx) / (prob.nx - 1)
    om = np.broadcast_to(np.exp(c * xi)[None, :], (prob.ny, prob.nx)).copy()
    xs = (1 - np.exp(-c * xi)) / (1 - np.exp(-c))
    x0 = np.broadcast_to(xs[None, :], (prob.ny, prob.nx)).copy()
    _, y0 = W.identity_mesh(prob)
    inp = prepared(prob, om, x0, y0)
    for (i0, j0) in [(32, 32), (16, 32), (48, 32)]:
        pos = (x0[j0, i0], y0[j0, i0])
        mean, se, _ = node_mean(inp, i0, j0, 100000, shift=pos)
        assert np.all(np.abs(mean - pos) < 4 * se + 2e-5), (mean, pos, se)
        omega = np.exp(c * xi[i0])
        drift_free = prob.dt / prob.tau * omega * c * c * np.exp(-c * xi[i0]) / (1 - np.exp(-c))
        if form == W.FORM_WINSLOW:
            drift_free /= omega
        assert drift_free > 20 * se[0]


# ---------------------------------------------------------------------------------------
# Hand-traced paths: constant omega, so phi^{k+1} = phi^k + sqrt(2 D ds) z^k exactly.
# ---------------------------------------------------------------------------------------

def test_hand_traced_paths_follow_counter_layout(oracle_lib):
    from test_oracle_philox import philox
    prob = make(nx=3, K=6, dt=0.03, tau=1.0, seed=0x1234_0000_0042)
    om = np.full((3, 3), 2.0)
    inp = prepared(prob, om, tstep=7)
    D = 2.0
    ds = prob.dt / prob.substeps
    key = np.array([0x0000_0042, 0x1234], np.uint32)
    m, i0, j0 = 3, 1, 1
    for p in range(4):
        val, steps, side, _ = mc.paths(inp, m, i0, j0, p, 1)
        phi = np.array([0.5, 0.5])
        exp_side, exp_steps = 4, prob.substeps
        for k in range(prob.substeps):
            w = philox([k, p, m, 7], key)[0]
            u1, u2, ub = ((w.astype(np.float64) + 0.5) * 2.0 ** -32)[:3]
            r = math.sqrt(-2 * math.log(u1))
            z = np.array([r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)])
            new = phi + math.sqrt(2 * D * ds) * z
            out = np.array([-new[0], new[0] - 1, -new[1], new[1] - 1])
            if out.max() > 0:
                exp_side, exp_steps = int(np.argmax(out)), k + 1
                break
            d0 = np.array([phi[0], 1 - phi[0], phi[1], 1 - phi[1]])
            d1 = np.array([new[0], 1 - new[0], new[1], 1 - new[1]])
            pr = np.exp(-d0 * d1 / (D * ds))
            if ub > np.prod(1 - pr):
                exp_side, exp_steps = int(np.argmax(pr)), k + 1
                break
            phi = new
        assert (side[0], steps[0]) == (exp_side, exp_steps)
        if exp_side == 4:
            assert np.allclose(val[0], phi, atol=1e-14)
        else:
            e = np.clip(new, 0, 1)
            e[exp_side // 2] = float(exp_side % 2)
            assert np.allclose(val[0], e, atol=1e-14)


# ---------------------------------------------------------------------------------------
# Estimator and adaptive path counts.
# ---------------------------------------------------------------------------------------

def test_estimate_matches_numpy_moments():
    rng = np.random.default_rng(8)
    v = rng.normal(3.0, 0.2, size=(7, 2, 1000))
    shift = np.array([[3.1, 2.9]] * 7)
    d = v - shift[:, :, None]
    sums = np.stack([d[:, 0].sum(1), (d[:, 0] ** 2).sum(1), d[:, 1].sum(1), (d[:, 1] ** 2).sum(1)], 1)
    mean, var, se = mc.estimate(sums, np.full(7, 1000), shift)
    assert np.allclose(mean, v.mean(axis=2), atol=1e-13)
    assert np.allclose(var, v.var(axis=2, ddof=1), rtol=1e-10)
    assert np.allclose(se, np.sqrt(v.var(axis=2, ddof=1) / 1000), rtol=1e-10)


def test_next_total_schedule():
    assert mc.next_total(4096, 1e-4, 1e-4, 10 ** 7) == 4096
    assert mc.next_total(4096, 2e-4, 1e-4, 10 ** 7) == int(math.ceil(4096 * 4 * 1.03 / 1024) * 1024)
    assert mc.next_total(4096, 1.01e-4, 1e-4, 10 ** 7) == 4096 + 1024
    assert mc.next_total(4096, 1.0, 1e-4, 50000) == 50000
    assert mc.next_total(50000, 1.0, 1e-4, 50000) == 50000
    for n in (1000, 3000, 70000):
        t = mc.next_total(n, 3e-4, 1e-4, 10 ** 8)
        assert t % 1024 == 0 and t > n


def test_adaptive_mc_reaches_target_and_is_independent_of_the_batch(oracle_lib):
    prob = W.c0_small_fp64().replace(paths_per_node=2048, se_target=4e-3, max_paths_per_node=200000)
    x, y = W.identity_mesh(prob)
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    om = monitor_on_mesh(prob, x, y, 0.0)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py)
    est, se, n_used, steps = mc.interface_mc(prob, x, y, om, nodes, 0)
    assert np.all(se.max(axis=1) <= prob.se_target)
    assert n_used.max() > prob.paths_per_node
    # node 5 alone: same ids, same counter streams, same chunk schedule -> identical result
    inp = mc.prepare(prob, x, y, om, 0)
    r = 5
    shift = [x[nodes[r, 1], nodes[r, 0]], y[nodes[r, 1], nodes[r, 0]]]
    n = prob.paths_per_node
    sums, _ = mc.interface_sums(inp, [r], nodes[r:r + 1], [0], [n], [shift])
    while True:
        _, _, s1 = mc.estimate(sums, np.array([n]), np.array([shift]))
        nt = mc.next_total(n, float(s1.max()), prob.se_target, prob.max_paths_per_node)
        if nt == n:
            break
        s2, _ = mc.interface_sums(inp, [r], nodes[r:r + 1], [n], [nt - n], [shift])
        sums += s2
        n = nt
    m1, _, _ = mc.estimate(sums, np.array([n]), np.array([shift]))
    assert n == n_used[r]
    assert np.array_equal(m1[0], est[r])
