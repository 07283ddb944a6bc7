"""Pins of the oracle's whole alternating step (Sec. 3.6)."""
import numpy as np
import pytest

import workloads as W
from oracle import step


@pytest.mark.parametrize("periodic", [0, 1])
def test_constant_monitor_keeps_the_uniform_mesh(periodic):
    """omega = 1 and the identity mesh: the exact step is the identity.  Interface estimates are
    within 4 SE of their nodes, and by the discrete maximum principle the subdomain interiors
    deviate from the identity by no more than the interface estimates do."""
    prob = W.Problem(name="t", nx=33, ny=33, px=2, py=2, periodic=periodic, tau=1e-2, dt=1e-3,
                     substeps=20, paths_per_node=4000, monitor_kind=W.MONITOR_BUMPS, monitor_params=[])
    x, y = W.identity_mesh(prob)
    r = step.step(prob, x, y, 0.0, 0)
    nodes = r["nodes"]
    pos = np.stack([x[nodes[:, 1], nodes[:, 0]], y[nodes[:, 1], nodes[:, 0]]], 1)
    dev = np.abs(r["est"] - pos)
    assert np.mean(dev < 4 * r["se"]) > 0.99
    bound = dev.max()
    assert np.abs(r["x"] - x).max() <= bound + 1e-12
    assert np.abs(r["y"] - y).max() <= bound + 1e-12
    assert np.all(r["n_used"] == prob.paths_per_node)


def test_c0_step_moves_nodes_toward_the_monitor_peak():
    """The Gaussian monitor attracts mesh lines toward its centre (equidistribution, Sec. 2)."""
    prob = W.c0_small_fp64()
    x, y = W.identity_mesh(prob)
    r = step.step(prob, x, y, 0.0, 0)
    xn = r["x"]
    assert np.all(np.isfinite(xn)) and np.all(np.isfinite(r["y"]))
    # along the middle row, nodes left of the centre move right and vice versa
    row = xn[16]
    xi = np.arange(33) / 32
    assert np.all(row[1:16] - xi[1:16] > 0) and np.all(row[17:32] - xi[17:32] < 0)
    # with N = 1000 paths the interface noise (SE ~ 1e-2) can fold a few of the compressed
    # cells next to the peak, but the bulk of the mesh stays ordered
    assert np.mean(np.diff(xn, axis=1) > 0) > 0.97 and np.mean(np.diff(r["y"], axis=0) > 0) > 0.97


def test_interface_sampling_keeps_node_streams_and_interpolates_the_rest():
    """With iface_stride > 1 the sampled nodes' estimates are those of the full evaluation (same
    node ids in the counter) and the others are the line interpolation of the sampled ones."""
    from oracle.layout import interface_nodes, interface_sampling
    from oracle.mc import interface_mc
    from oracle.step import monitor_on_mesh
    prob = W.c0_small_fp64().replace(nx=17, ny=17, paths_per_node=64)
    x, y = W.identity_mesh(prob)
    om = monitor_on_mesh(prob, x, y, 0.0)
    nodes = interface_nodes(17, 17, 2, 2)
    e1, s1, n1, _ = interface_mc(prob, x, y, om, nodes, 0)
    samp = prob.replace(iface_stride=3)
    e3, s3, n3, _ = interface_mc(samp, x, y, om, nodes, 0)
    mask, fill = interface_sampling(17, 17, 2, 2, 0, 3)
    assert np.array_equal(e3[mask], e1[mask]) and np.array_equal(n3[mask], n1[mask])
    assert np.all(n3[~mask] == 0) and np.all(s3[~mask] == 0)
    blank = e3.copy()
    blank[~mask] = np.nan
    assert np.array_equal(fill(blank), e3)


def test_mkp_with_one_submesh_is_the_plain_step():
    from oracle.step import mkp_step
    prob = W.c0_small_fp64().replace(nx=17, ny=17, paths_per_node=32)
    x, y = W.identity_mesh(prob)
    a = step.step(prob, x, y, 0.0, 3)
    b = mkp_step(prob, x, y, 0.0, 3, 1)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])


def test_mkp_with_a_static_monitor_is_plain_steps_of_dt_over_k():
    """A nodal monitor depends on neither time nor position, so freezing it at t^n changes
    nothing: K sub-meshes equal K plain steps of dt/K with counter words n K + k."""
    from oracle.step import mkp_step
    prob = W.c0_small_fp64().replace(nx=17, ny=17, paths_per_node=32, monitor_kind=W.MONITOR_NODAL,
                                     monitor_params=[])
    x, y = W.sine_mode_mesh(prob, amp=0.02)
    om = 1.0 + 0.3 * np.sin(np.pi * x) ** 2
    K, n = 3, 2
    r = mkp_step(prob, x, y, 0.0, n, K, omega_nodal=om)
    sub = prob.replace(dt=prob.dt / K)
    xs, ys = x, y
    for k in range(K):
        q = step.step(sub, xs, ys, 123.0, n * K + k, omega_nodal=om)
        xs, ys = q["x"], q["y"]
    assert np.array_equal(r["x"], xs) and np.array_equal(r["y"], ys)
