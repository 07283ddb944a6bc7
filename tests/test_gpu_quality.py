"""Mesh quality on the GPU (Eq. 8) and the paper's periodic five-ring experiment (Sec. 4.2):
100 SDD steps on 41 x 41 nodes with 2 x 2, 3 x 3 and 4 x 4 subdomains against the single-domain
reference mesh (the paper reports R_max = R_mean = 1), and in the paper's one-substep setting
against the oracle's own SDD trajectory."""
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


def _single_domain_reference(prob):
    xs, ys = W.identity_mesh(prob)
    for n in range(prob.steps):
        om = monitor_on_grid(prob.monitor_kind, prob.monitor_params, xs, ys, n * prob.dt, 1, prob.Lx, prob.Ly)
        xs, ys = periodic_single_domain_step(om, xs, ys, prob.dt, prob.tau, prob.form, prob.Lx, prob.Ly)
    return cell_quality(xs, ys)


def _five_ring_gpu(prob, keep=()):
    h = gpu_problem(prob)
    kept = {}
    for s in range(1, prob.steps + 1):
        h.step()
        if s in keep:
            kept[s] = h.mesh()
    gx, gy = h.mesh()
    q_gpu, _, _ = h.quality()
    h.close()
    q_sdd = cell_quality(gx, gy)
    assert np.allclose(q_gpu, q_sdd, rtol=1e-12)
    return q_sdd, kept


@pytest.mark.parametrize("px", [2, 3, 4])
def test_five_ring_resolved_substeps_quality_ratio(px):
    """Sixteen Euler-Maruyama substeps per step: the paper's R_max = R_mean = 1 to two digits
    (R_max read as max Q_SD / max Q_SDD; the largest per-cell ratio stays below 1.1)."""
    prob = W.five_ring(px).replace(substeps=16)
    q_sdd, _ = _five_ring_gpu(prob)
    q_sd = _single_domain_reference(prob)
    r = ratio_stats(q_sd, q_sdd)
    print(f"five-ring {px}x{px} K=16: {r} Q_SD max {q_sd.max():.3f} Q_SDD max {q_sdd.max():.3f}")
    assert q_sd.max() > 1.2  # the mesh adapted: cells concentrate at the rings
    assert 0.99 <= r["R_mean"] <= 1.01
    assert 0.98 <= r["maxQ_ratio"] <= 1.02
    assert r["R_max"] <= 1.1


@pytest.mark.parametrize("px", [2, 3, 4])
def test_five_ring_paper_setting_is_the_oracle_trajectory(px):
    """The paper's own setting, one Euler-Maruyama substep per step (ds = dt), 100 steps.

    The GPU's SDD trajectory is the oracle's SDD trajectory on the same Philox streams: meshes
    within 1e-6 after steps 1, 10 and 100, and the final quality ratios against the single-domain
    reference equal to the oracle's (max-Q ratio to 1e-4 relative, mean R to 1e-6).  The mean ratio R stays within 3 % of 1 (the paper's
    R_mean = 1); the max-Q ratio does not reach the paper's 1 in either implementation.  Cause
    (the method at this resolution, not the kernel): with one substep an interface estimate is
    the explicit drift step xi + (grad omega / omega) dt, which moves nodes at the rings by up
    to 1.5 cells while dt |d b / d xi| = 1.2, so neighbouring interface nodes overshoot the
    implicit single-domain solution by up to 0.7 cell and a few cells fold (tested on the
    oracle alone in test_oracle_quality.py)."""
    from oracle import step as ostep
    prob = W.five_ring(px)
    keep = (1, 10, 100)
    q_sdd, kept = _five_ring_gpu(prob, keep)
    x, y = W.identity_mesh(prob)
    for n in range(prob.steps):
        r = ostep.step(prob, x, y, prob.t0 + n * prob.dt, n)
        x, y = r["x"], r["y"]
        if n + 1 in keep:
            gx, gy = kept[n + 1]
            assert max(np.abs(gx - x).max(), np.abs(gy - y).max()) <= 1e-6
    q_oracle = cell_quality(x, y)
    q_sd = _single_domain_reference(prob)
    r_gpu = ratio_stats(q_sd, q_sdd)
    r_or = ratio_stats(q_sd, q_oracle)
    print(f"five-ring {px}x{px} K=1: gpu {r_gpu} oracle {r_or}")
    # the worst cells are nearly folded (Q up to ~1e2..1e4), so Q amplifies the meshes' 1e-8
    # differences: the ratios agree to 1e-4 relative
    assert abs(r_gpu["maxQ_ratio"] - r_or["maxQ_ratio"]) <= 1e-4 * r_or["maxQ_ratio"]
    assert abs(r_gpu["R_mean"] - r_or["R_mean"]) <= 1e-6
    assert 0.97 <= r_gpu["R_mean"] <= 1.03
