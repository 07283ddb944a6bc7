"""Invalid inputs found on the device: a monitor that is not finite and positive at every node
(omega > 0 is required by Sec. 2) makes the interface Monte Carlo, the step, a batch step and a
served request report SDD_ERR_INVALID_ARG; no step is taken, and the problem stays usable."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem
from test_gpu_batch import small_mix
from test_gpu_serving import alone, drain, server_params, submit

pytestmark = pytest.mark.gpu


def nodal_case():
    return W.c0_small_fp64().replace(precision=W.PREC_FP32_KAHAN, monitor_kind=W.MONITOR_NODAL,
                                     monitor_params=[], paths_per_node=2048)


@pytest.mark.parametrize("bad_value", [np.nan, np.inf, 0.0, -1.0])
def test_invalid_monitor_rejected_and_problem_reusable(bad_value):
    import paper_1504_00084_gb300 as S
    prob = nodal_case()
    x, y = W.identity_mesh(prob)
    om = 1.0 + 0.5 * np.sin(3 * x) ** 2
    bad = om.copy()
    bad[7, 9] = bad_value
    h = gpu_problem(prob)
    h.set_monitor(bad)
    with pytest.raises(S.SddError) as e:
        h.interface_mc()
    assert e.value.status == S.SDD_ERR_INVALID_ARG
    with pytest.raises(S.SddError) as e:
        h.step()
    assert e.value.status == S.SDD_ERR_INVALID_ARG
    gx, gy = h.mesh()
    assert np.array_equal(gx, x) and np.array_equal(gy, y)  # no step taken
    assert h.stats()["step_index"] == 0
    h.set_monitor(om)
    h.step()
    ref = gpu_problem(prob, omega=om)
    ref.step()
    rx, ry = ref.mesh()
    gx, gy = h.mesh()
    assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
    h.close()
    ref.close()


def test_batch_reports_invalid_monitor():
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=3)
    hs = [gpu_problem(p) for p in probs]
    bad = np.full((probs[1].ny, probs[1].nx), 1.0)
    bad[3, 3] = np.nan
    hs[1].set_monitor(bad)
    with S.SddBatch(hs, stream=torch.cuda.Stream()) as b:
        b.step()
        with pytest.raises(S.SddError) as e:
            b.stats()
        assert e.value.status == S.SDD_ERR_INVALID_ARG
    for h in hs:
        h.close()


def test_server_reports_invalid_request_and_serves_the_others():
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=3, se_target=6e-3)
    refs = [alone(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, 6e-3, 1 << 16), stream) as srv:
        ids = [submit(srv, p) for p in probs]
        q = probs[0].replace(seed=4242)
        x, y = W.identity_mesh(q)
        om = np.full((q.ny, q.nx), 2.0)
        om[5, 5] = -3.0
        bad_id = srv.submit(S.params_from(q), x, y, S.SDD_MONITOR_NODAL, None, omega=om)
        drain(srv, len(ids) + 1)
        with pytest.raises(S.SddError) as e:
            srv.result(bad_id)
        assert e.value.status == S.SDD_ERR_INVALID_ARG
        for rid, (rx, ry, rest, _) in zip(ids, refs):
            out = srv.result(rid)
            assert np.array_equal(out["x"], rx) and np.array_equal(out["y"], ry)
