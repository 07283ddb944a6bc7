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
