"""A time step split by interface nodes (sdd_interface_mc_range, then sdd_step_from_interface).
The estimate at a node depends on that node's own paths only (Sec. 3.4: the Philox counter
carries the node id), so the ranges of a partition of [0, M), computed apart and assembled, give
bitwise the estimates and the new mesh of sdd_step.  This is the exchange of a problem shared by
several GPUs (one allgather of M x 2 estimates); here the ranges run one after another on one GPU,
over two steps, with ragged ranges, fixed and adaptive path counts."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem

pytestmark = pytest.mark.gpu


def _problem(precision, adaptive):
    prob = W.c0_small_fp64().replace(precision=precision, px=3, py=2, paths_per_node=3000)
    if adaptive:
        prob = prob.replace(se_target=2e-3, paths_per_node=2048, max_paths_per_node=1 << 16)
    return prob


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("precision,adaptive", [(W.PREC_FP64, False), (W.PREC_FP32_KAHAN, False),
                                                (W.PREC_FP32_KAHAN, True)])
def test_node_ranges_assemble_to_the_full_step(precision, adaptive, parts):
    prob = _problem(precision, adaptive)
    x, y = W.sine_mode_mesh(prob, amp=0.02)
    ref = gpu_problem(prob, x, y)
    split = gpu_problem(prob, x, y)
    M = ref.M
    bounds = [0] + [int(round(M * k / parts)) + (k % 2) for k in range(1, parts)] + [M]  # ragged
    for _ in range(2):
        rest, rse, rn, _ = ref.interface_mc()
        rx, ry, _ = ref.step()
        est = np.full((M, 2), np.nan)
        se = np.full((M, 2), np.nan)
        n = np.full(M, -1, dtype=np.int64)
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            before = est.copy()
            split.interface_mc_range(lo, hi, est, se, n)
            assert np.array_equal(np.delete(est, np.s_[lo:hi], axis=0), np.delete(before, np.s_[lo:hi], axis=0),
                                  equal_nan=True)  # only the range's rows written
        assert np.array_equal(est, rest) and np.array_equal(se, rse) and np.array_equal(n, rn)
        gx, gy, _ = split.step_from_interface(est)
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
    assert split.stats()["step_index"] == ref.stats()["step_index"] == 2
    ref.close()
    split.close()


def test_node_range_rejections():
    import paper_1504_00084_gb300 as S
    prob = _problem(W.PREC_FP64, False)
    h = gpu_problem(prob)
    M = h.M
    for lo, hi in [(-1, 3), (4, 3), (0, M + 1)]:
        with pytest.raises(S.SddError) as e:
            h.interface_mc_range(lo, hi)
        assert e.value.status == S.SDD_ERR_INVALID_ARG
    est, _, n, st = h.interface_mc_range(5, 5)  # empty range: nothing computed or written
    assert st == S.SDD_OK and not est.any() and not n.any()
    h.close()
    sampled = gpu_problem(prob.replace(nx=65, ny=65, px=2, py=2, iface_stride=4))
    with pytest.raises(S.SddError) as e:
        sampled.interface_mc_range(0, 3)
    assert e.value.status == S.SDD_ERR_INVALID_ARG
    sampled.close()
