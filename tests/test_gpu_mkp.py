"""M^kP steps (sdd_step_mkp, Sec. 5): K = 1 is bitwise the plain step; K sub-meshes match the
oracle's M^kP step (monitor re-evaluated on every sub-mesh at the step's time, counter words
n K + k) within the FP64 mesh tolerance; the step index and time advance by one step."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem
from oracle import step as ostep
from gpu_helpers import mesh_tolerance

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32_KAHAN])
def test_mkp_one_submesh_is_plain_step(precision):
    prob = W.c0_small_fp64().replace(precision=precision, paths_per_node=2048)
    a = gpu_problem(prob)
    b = gpu_problem(prob)
    for _ in range(2):
        ax, ay, _ = a.step()
        bx, by, _ = b.step_mkp(1)
    assert np.array_equal(ax, bx) and np.array_equal(ay, by)
    assert b.stats()["step_index"] == 2
    a.close()
    b.close()


@pytest.mark.parametrize("monitor", ["gauss", "front"])
def test_mkp_matches_oracle_fp64(monitor):
    prob = W.c0_small_fp64()
    if monitor == "front":
        # moving front: freezing the monitor time at t^n matters
        prob = prob.replace(monitor_kind=W.MONITOR_FRONT, monitor_params=[2.0, 4.0, 0.25, 5.0, 0.5, 0.5])
    K = 3
    x, y = W.identity_mesh(prob)
    h = gpu_problem(prob, x, y)
    h.step()                          # step 0 (plain), then an M^kP step from step index 1
    x1, y1 = h.mesh()
    gx, gy, _ = h.step_mkp(K)
    r0 = ostep.step(prob, x, y, prob.t0, 0)
    ox1, oy1 = r0["x"], r0["y"]
    tol1 = mesh_tolerance(prob, r0["omega"], *ostep.scatter(prob, r0["nodes"], r0["est"]), x, y, 1e-10)
    assert np.abs(x1 - ox1).max() <= tol1 and np.abs(y1 - oy1).max() <= tol1
    r = ostep.mkp_step(prob, x1, y1, prob.t0 + prob.dt, 1, K)
    sub = prob.replace(dt=prob.dt / K)
    bx, by = ostep.scatter(sub, r["nodes"], r["est"])
    tol = K * 2 * mesh_tolerance(sub, r["omega"], bx, by, x1, y1, 1e-10)
    assert np.abs(gx - r["x"]).max() <= tol and np.abs(gy - r["y"]).max() <= tol
    st = h.stats()
    assert st["step_index"] == 2 and abs(st["t"] - (prob.t0 + 2 * prob.dt)) < 1e-15
    h.close()
