"""Batches of independent problems (sdd_batch_*): every problem's mesh after batched steps is
bitwise the mesh of stepping it alone, in plain and CUDA-graph mode, for uneven grids and
splits, mixed boundary kinds and generator forms, fixed and adaptive path counts."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem

pytestmark = pytest.mark.gpu


def small_mix(precision, paths=4096, n=6, se_target=0.0):
    """Shapes and bump monitors of the batched-mix workload, shrunk to test size."""
    base = W.c3_mix(n, paths=paths)
    out = []
    for k, p in enumerate(base):
        nx = 33 if p.nx <= 129 else 65
        split = min(p.px, (nx - 1) // 4)
        q = p.replace(nx=nx, ny=nx, px=split, py=split, precision=precision, paths_per_node=paths,
                      se_target=se_target, max_paths_per_node=(1 << 16) if se_target > 0 else 0)
        if k % 3 == 1:
            q = q.replace(periodic=1)
        if k % 3 == 2:
            q = q.replace(form=W.FORM_WINSLOW, tau=0.1)
        out.append(q)
    return out


def meshes_alone(probs, steps):
    res = []
    for prob in probs:
        h = gpu_problem(prob)
        for _ in range(steps):
            h.step()
        res.append(h.mesh())
        h.close()
    return res


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("precision", [W.PREC_FP32_KAHAN, W.PREC_FP64])
def test_batch_bitwise_equals_problems_alone(use_graph, precision):
    import torch

    import paper_1504_00084_gb300 as S
    paths = 4096 if precision != W.PREC_FP64 else 1024
    probs = small_mix(precision, paths=paths)
    steps = 3
    ref = meshes_alone(probs, steps)
    stream = torch.cuda.Stream()
    hs = [gpu_problem(p) for p in probs]
    with S.SddBatch(hs, stream=stream, use_graph=use_graph) as b:
        for _ in range(steps):
            b.step()
        st = b.stats()
    stream.synchronize()
    assert st["M"] == sum(h.M for h in hs)
    assert st["paths"] == st["M"] * paths
    for h, (rx, ry) in zip(hs, ref):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        assert h.stats()["step_index"] == steps
        h.close()


def test_adaptive_batch_bitwise_equals_problems_alone():
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, se_target=6e-3)
    ref = meshes_alone(probs, 2)
    hs = [gpu_problem(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddBatch(hs, stream=stream) as b:
        b.step()
        b.step()
        st = b.stats()
    assert st["mc_rounds"] >= 2 and st["nodes_not_reached"] == 0
    for h, (rx, ry) in zip(hs, ref):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        h.close()


def test_batch_rejects_mixed_settings():
    import paper_1504_00084_gb300 as S
    a = gpu_problem(W.c0_small_fp64())
    b = gpu_problem(W.c0_small_fp64().replace(precision=W.PREC_FP32_KAHAN))
    with pytest.raises(S.SddError):
        S.SddBatch([a, b])
    with pytest.raises(S.SddError):
        S.SddBatch([a, a])
    with pytest.raises(S.SddError):
        S.SddBatch([a], stream=None, use_graph=True)   # graph mode needs a stream
    a.close(); b.close()


def test_batch_mixing_subdomain_schemes_equals_alone():
    """Forward-Euler problems (the paper's local solver) and backward-Euler ones in one batch."""
    import torch

    import paper_1504_00084_gb300 as S
    probs = [p.replace(subdomain_scheme=k % 2) for k, p in enumerate(small_mix(W.PREC_FP32_KAHAN, paths=2048, n=4))]
    ref = meshes_alone(probs, 1)
    hs = [gpu_problem(p) for p in probs]
    with S.SddBatch(hs, stream=torch.cuda.Stream()) as b:
        b.step()
        st = b.stats()
    assert st["solve_iters_max"] >= 1
    for h, (rx, ry) in zip(hs, ref):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        h.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_block_size_tuning_keeps_results(use_graph):
    """sdd_batch_tune: the path-kernel block size (128, 256 or 512 threads, or tuned by timing all
    three on the next step's first round) never changes results: every size gives bitwise the
    meshes of stepping each problem alone, tuning itself changes no problem's state, and an
    unsupported size is rejected."""
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=4096, n=4)
    steps = 3
    ref = meshes_alone(probs, steps)
    stream = torch.cuda.Stream()
    hs = [gpu_problem(p) for p in probs]
    with S.SddBatch(hs, stream=stream, use_graph=use_graph) as b:
        assert b.tune(0) in (128, 256, 512)
        for tpb in (128, 512, 256):
            assert b.tune(tpb) == tpb
            b.step()
        with pytest.raises(S.SddError):
            b.tune(96)
        b.stats()
    stream.synchronize()
    for h, (rx, ry) in zip(hs, ref):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        h.close()
