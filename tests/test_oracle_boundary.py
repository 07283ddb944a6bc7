"""Pins of the moving physical boundary (Sec. 2): the 1-D generator step along a side, and the
exit values of paths when the boundary mesh is not the identity."""
import math

import numpy as np

import workloads as W
from oracle import mc
from oracle.boundary import boundary_mesh_step, side_step
from oracle.layout import interface_nodes
from oracle.step import monitor_on_mesh


def test_uniform_side_with_constant_monitor_is_kept():
    b = np.linspace(0.0, 2.0, 17)
    assert np.allclose(side_step(np.full(17, 3.0), b, 0.7, 0), b, atol=1e-15)
    assert np.allclose(side_step(np.full(17, 3.0), b, 0.7, 1), b, atol=1e-15)


def test_side_mode_decay_closed_form():
    """Constant omega: sin(pi k h) is an eigenvector of the 1-D operator with eigenvalue
    r w (4 / h^2) sin^2(pi h / 2); one backward-Euler step divides it by 1 + that."""
    n, w0, r, A = 33, 2.0, 3e-3, 0.01
    k = np.arange(n)
    h = 1.0 / (n - 1)
    base = k * h
    b = base + A * np.sin(np.pi * k * h)
    lam = r * w0 * (4 / h ** 2) * math.sin(math.pi * h / 2) ** 2
    got = side_step(np.full(n, w0), b, r, 0)
    assert np.allclose(got, base + A / (1 + lam) * np.sin(np.pi * k * h), atol=1e-15)


def test_side_steady_state_equidistributes():
    """r -> infinity: (w b_xi)_xi = 0, so b_{k+1} - b_k is proportional to 1 / (w_k + w_{k+1})."""
    rng = np.random.default_rng(3)
    n = 21
    w = rng.uniform(0.5, 4.0, n)
    b = np.linspace(0.0, 1.5, n)
    got = side_step(w, b, 1e13, 0)
    inv = 1.0 / (w[:-1] + w[1:])
    want = np.concatenate([[0.0], np.cumsum(inv)]) * 1.5 / inv.sum()
    assert np.allclose(got, want, atol=1e-10)


def test_identity_boundary_gives_the_fixed_boundary_exit_values():
    prob = W.c0_small_fp64().replace(nx=17, ny=17)
    x, y = W.identity_mesh(prob)
    om = monitor_on_mesh(prob, x, y, 0.0)
    bnd = np.concatenate([x[0, :], x[-1, :], y[:, 0], y[:, -1]])
    nodes = interface_nodes(17, 17, 2, 2)
    a = mc.paths(mc.prepare(prob, x, y, om, 0), 3, int(nodes[3, 0]), int(nodes[3, 1]), 0, 400)
    b = mc.paths(mc.prepare(prob, x, y, om, 0, bnd=bnd), 3, int(nodes[3, 0]), int(nodes[3, 1]), 0, 400)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.allclose(a[0], b[0], atol=1e-15, rtol=0)


def test_moving_boundary_step_adapts_the_boundary():
    """With a monitor peaked at the domain centre the bottom side's nodes move toward its
    middle; the normal components and the corners stay put."""
    prob = W.c0_small_fp64().replace(nx=33, ny=33, moving_boundary=1, dt=1.0)
    x, y = W.identity_mesh(prob)
    om = monitor_on_mesh(prob, x, y, 0.0)
    bnd = boundary_mesh_step(prob, om, x, y)
    bottom = bnd[:33]
    assert bottom[0] == 0.0 and bottom[-1] == prob.Lx
    assert np.all(np.diff(bottom) > 0)
    gaps = np.diff(bottom)
    assert gaps[15] < gaps[0]   # finer cells near the monitor peak at x = 1/2
