"""Mesh quality on the GPU (Eq. 8) and the paper's periodic five-ring experiment (Sec. 4.2):
100 SDD steps on 41 x 41 nodes with 2 x 2 and 4 x 4 subdomains against the single-domain
reference mesh; the paper reports R_max = R_mean = 1."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem
from oracle.monitor import fd_gradient, monitor_on_grid
from oracle.quality import cell_quality, ratio_stats
from oracle.solve import periodic_single_domain_step

pytestmark = pytest.mark.gpu


def test_quality_kernel_matches_oracle():
    prob = W.c0_small_fp64()
    x, y = W.sine_mode_mesh(prob, amp=0.05)
    rng = np.random.default_rng(3)
    x[1:-1, 1:-1] += 0.004 * rng.normal(size=(31, 31))
    y[1:-1, 1:-1] += 0.004 * rng.normal(size=(31, 31))
    h = gpu_problem(prob, x, y)
    q, qmax, qmean = h.quality()
    ref = cell_quality(x, y)
    assert np.allclose(q, ref, rtol=1e-13)
    assert abs(qmax - ref.max()) <= 1e-13 * ref.max() and abs(qmean - ref.mean()) <= 1e-12
    h.close()


def test_ring_monitor_parity():
    prob = W.five_ring(2)
    x, y = W.sine_mode_mesh(prob, amp=0.02, periodic_mode=True)
    h = gpu_problem(prob, x, y)
    w, wx, we = h.monitor()
    om = monitor_on_grid(prob.monitor_kind, prob.monitor_params, x, y, 0.0, 1, prob.Lx, prob.Ly)
    gx, gy = fd_gradient(om, 1)
    assert np.abs(w - om).max() <= 1e-13 * om.max()
    assert np.abs(wx - gx).max() <= 1e-12 * np.abs(gx).max() and np.abs(we - gy).max() <= 1e-12 * np.abs(gy).max()
    h.close()


def _five_ring(px, substeps):
    prob = W.five_ring(px).replace(substeps=substeps)
    x, y = W.identity_mesh(prob)
    h = gpu_problem(prob, x, y)
    for _ in range(prob.steps):
        h.step()
    gx, gy = h.mesh()
    q_gpu, _, _ = h.quality()
    h.close()
    q_sdd = cell_quality(gx, gy)
    assert np.allclose(q_gpu, q_sdd, rtol=1e-12)
    xs, ys = x, y
    for n in range(prob.steps):
        om = monitor_on_grid(prob.monitor_kind, prob.monitor_params, xs, ys, n * prob.dt, 1, prob.Lx, prob.Ly)
        xs, ys = periodic_single_domain_step(om, xs, ys, prob.dt, prob.tau, prob.form, prob.Lx, prob.Ly)
    q_sd = cell_quality(xs, ys)
    r = ratio_stats(q_sd, q_sdd)
    print(f"five-ring {px}x{px} K={substeps}: {r} Q_SD max {q_sd.max():.3f} Q_SDD max {q_sdd.max():.3f}")
    assert q_sd.max() > 1.2  # the mesh adapted: cells concentrate at the rings
    return r


@pytest.mark.parametrize("px", [2, 3, 4])
@pytest.mark.parametrize("substeps", [1, 16])
def test_five_ring_quality_ratio(px, substeps):
    """Paper's setting is one Euler-Maruyama substep per step.  The rings are resolved by about
    one cell (the monitor jumps from 1 to 9.5 within a cell), so a single substep carries a
    drift of several cells evaluated at its start point: the interface estimates are biased
    near the rings, and a few cells there come out much worse than in the single-domain mesh
    although the mean ratio stays at 1.  Sixteen substeps remove most of that bias."""
    r = _five_ring(px, substeps)
    assert 0.97 <= r["R_mean"] <= 1.03
    if substeps >= 16:   # the paper's R_max = R_mean = 1 (two digits; R_max read as max Q_SD / max Q_SDD)
        assert 0.99 <= r["R_mean"] <= 1.01
        assert 0.98 <= r["maxQ_ratio"] <= 1.02
        assert r["R_max"] <= 1.1
