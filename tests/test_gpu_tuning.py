"""Launch configuration of the path kernel and its autotuner (sdd_get/set_mc_config, sdd_tune,
sdd_batch_get/set_mc_config, sdd_batch_tune_mc).  Threads per block and resident blocks per SM
never change a result (bitwise); the task size groups the estimator sums differently, so FP64
estimates stay within rounding of each other and of the oracle, and a batch gives bitwise the
results of its problems stepped alone with the same task size."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem, oracle_inputs
from oracle import mc

pytestmark = pytest.mark.gpu


def _estimates(prob, **cfg):
    h = gpu_problem(prob)
    if cfg:
        h.set_mc_config(**cfg)
    est, se, n, _ = h.interface_mc()
    st = h.stats()
    c = h.mc_config()
    h.close()
    return est, se, n, st["path_steps"], c


@pytest.mark.parametrize("adaptive", [False, True])
def test_blocks_per_sm_keep_results_bitwise(adaptive):
    prob = W.c0_small_fp64().replace(precision=W.PREC_FP32_KAHAN, paths_per_node=6000)
    if adaptive:
        prob = prob.replace(paths_per_node=2048, se_target=4e-3, max_paths_per_node=1 << 18)
    ref = _estimates(prob)
    assert ref[4]["threads_per_block"] == 256 and ref[4]["paths_per_task"] == 2048
    assert ref[4]["blocks_per_sm"] == ref[4]["max_blocks_per_sm"] >= 1
    for bps in range(1, ref[4]["max_blocks_per_sm"]):
        got = _estimates(prob, blocks_per_sm=bps)
        assert got[4]["blocks_per_sm"] == bps
        for a, b in zip(ref[:4], got[:4]):
            assert np.array_equal(a, b)


def test_task_size_changes_only_the_summation_grouping():
    """FP64, fixed N = 9000 (not a multiple of any task size): the same paths at every task size
    (identical path counts and substep totals), estimates within 1e-13 of each other and within
    1e-10 of the oracle's sequential sums.  Per-path records do not depend on the task size."""
    prob = W.c0_small_fp64().replace(paths_per_node=9000)
    x, y = W.identity_mesh(prob)
    om, inp, nodes = oracle_inputs(prob, x, y, prob.t0, 0)
    oest, ose, on, osteps = mc.interface_mc(prob, x, y, om, nodes, 0, np.float64)
    base = None
    for tp in (1024, 2048, 4096):
        est, se, n, steps, c = _estimates(prob, paths_per_task=tp)
        assert c["paths_per_task"] == tp
        assert np.array_equal(n, on) and steps == int(osteps.sum())
        assert np.abs(est - oest).max() <= 1e-10 and np.abs(se - ose).max() <= 1e-10
        if base is None:
            base = (est, se)
        assert np.abs(est - base[0]).max() <= 1e-13 and np.abs(se - base[1]).max() <= 1e-13
    h = gpu_problem(prob)
    h.set_mc_config(paths_per_task=4096)
    v, s_, d = h.debug_paths(7, 0, 5000)
    h.close()
    ov, os_, od, _ = mc.paths(inp, 7, int(nodes[7, 0]), int(nodes[7, 1]), 0, 5000)
    assert np.array_equal(s_, os_) and np.array_equal(d, od) and np.abs(v - ov).max() <= 1e-12


def test_invalid_configurations_are_rejected():
    import paper_1504_00084_gb300 as S
    h = gpu_problem(W.c0_small_fp64())
    c = h.mc_config()
    for kw in ({"threads_per_block": 128}, {"blocks_per_sm": c["max_blocks_per_sm"] + 1},
               {"blocks_per_sm": -1}, {"paths_per_task": 3000}, {"paths_per_task": 512}):
        with pytest.raises(S.SddError):
            h.set_mc_config(**kw)
    assert h.mc_config() == c
    h.close()


def test_tune_keeps_state_and_picks_a_listed_configuration():
    """sdd_tune changes no state: the step after tuning is bitwise the step of a fresh problem
    given the chosen configuration explicitly."""
    prob = W.c1_front(W.PREC_FP32_KAHAN).replace(nx=129, ny=129, paths_per_node=20000, se_target=0.0,
                                                 max_paths_per_node=20000)
    h = gpu_problem(prob)
    chosen = h.tune_mc(True)
    assert chosen["threads_per_block"] == 256 and chosen["paths_per_task"] in (1024, 2048, 4096)
    assert 1 <= chosen["blocks_per_sm"] <= chosen["max_blocks_per_sm"]
    gx, gy, _ = h.step()
    assert h.stats()["step_index"] == 1
    h.close()
    h2 = gpu_problem(prob)
    h2.set_mc_config(blocks_per_sm=chosen["blocks_per_sm"], paths_per_task=chosen["paths_per_task"])
    rx, ry, _ = h2.step()
    h2.close()
    assert np.array_equal(gx, rx) and np.array_equal(gy, ry)


@pytest.mark.parametrize("tune", [False, True])
def test_batch_configuration_keeps_results_of_problems_alone(tune):
    """A batch with a set (or tuned) configuration: every problem's mesh after two batched steps
    is bitwise the mesh of stepping it alone with the batch's task size (block size and blocks
    per SM do not matter)."""
    import torch

    import paper_1504_00084_gb300 as S
    from test_gpu_batch import small_mix
    probs = small_mix(W.PREC_FP32_KAHAN, paths=4096, n=4)
    hs = [gpu_problem(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddBatch(hs, stream=stream) as b:
        if tune:
            cfg = b.tune_mc(True)
        else:
            b.set_mc_config(threads_per_block=512, blocks_per_sm=1, paths_per_task=4096)
            cfg = b.mc_config()
            assert (cfg["threads_per_block"], cfg["blocks_per_sm"], cfg["paths_per_task"]) == (512, 1, 4096)
        assert all(h.mc_config()["paths_per_task"] == cfg["paths_per_task"] for h in hs)
        b.step()
        b.step()
        b.stats()
    stream.synchronize()
    for prob, h in zip(probs, hs):
        gx, gy = h.mesh()
        h.close()
        a = gpu_problem(prob)
        a.set_mc_config(paths_per_task=cfg["paths_per_task"])
        a.step()
        rx, ry, _ = a.step()
        a.close()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)


def test_batch_rejects_mixed_task_sizes():
    import paper_1504_00084_gb300 as S
    a = gpu_problem(W.c0_small_fp64())
    b = gpu_problem(W.c0_small_fp64().replace(seed=5))
    b.set_mc_config(paths_per_task=1024)
    with pytest.raises(S.SddError):
        S.SddBatch([a, b])
    a.close(); b.close()
