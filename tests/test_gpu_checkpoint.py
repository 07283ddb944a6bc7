"""Checkpoint / resume (sdd_save, sdd_load): a problem saved after some steps and resumed in a
new problem continues bit for bit as the original (the only random state is the Philox
counter's time-step word, which the checkpoint carries)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["front_adaptive", "nodal_periodic", "fp64"])
def test_resume_continues_bitwise(case, tmp_path):
    import paper_1504_00084_gb300 as S
    omega = None
    if case == "front_adaptive":
        prob = W.c1_front(W.PREC_FP32_KAHAN).replace(nx=65, ny=65, paths_per_node=2048, se_target=3e-3,
                                                     max_paths_per_node=1 << 16)
    elif case == "nodal_periodic":
        prob = W.c0_small_fp64().replace(precision=W.PREC_FP32_ACC64, periodic=1, monitor_kind=W.MONITOR_NODAL,
                                         monitor_params=[], paths_per_node=4096)
        x, y = W.identity_mesh(prob)
        omega = 1.0 + 0.5 * np.cos(2 * np.pi * x) ** 2
    else:
        prob = W.c0_small_fp64().replace(paths_per_node=1000)
    a = gpu_problem(prob, omega=omega)
    for _ in range(3):
        a.step()
    ra = a.mesh()
    b = gpu_problem(prob, omega=omega)
    b.step()
    path = str(tmp_path / "p.ckpt")
    b.save(path)
    b.close()
    c = S.SddProblem.load(path)
    assert c.stats()["step_index"] == 1
    c.step()
    c.step()
    rc = c.mesh()
    assert np.array_equal(ra[0], rc[0]) and np.array_equal(ra[1], rc[1])
    assert c.stats()["step_index"] == 3
    a.close()
    c.close()
