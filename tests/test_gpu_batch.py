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


def oracle_anchor_problems(paths=1000):
    """FP64 problems of uneven shapes for the oracle comparisons of batches and served requests:
    33 x 33 split 3 x 5 (subdomains of 10/11/11 by 6/6/7/6/7 cells, Gaussian monitor), a
    periodic 33 x 33 split 3 x 3 with the peak off centre at tau = 1, and the paper's generator
    form on a 25 x 25 grid split 2 x 3 at tau = 1.  (Periodic paths never exit: at tau = 1e-2
    their 100 substeps multiply a position difference by ~1e5, so a second step started from
    meshes that differ at 1e-10 would differ at 1e-5; at tau = 1 the factor stays near 1.)"""
    base = W.c0_small_fp64().replace(paths_per_node=paths)
    return [base.replace(px=3, py=5, seed=11),
            base.replace(px=3, py=3, periodic=1, tau=1.0, monitor_params=[6.0, 40.0, 0.3, 0.6], seed=12),
            base.replace(nx=25, ny=25, px=2, py=3, form=W.FORM_WINSLOW, tau=1.0, seed=13)]


def test_batch_fp64_matches_oracle():
    """Batched steps against the oracle itself: three FP64 problems of different grids, uneven
    splits, boundary kinds and generator forms in one batch (plus one of the bump-monitor mix),
    two steps.  After the first step every interface node's new position (its estimate) is the
    oracle's within 1e-10, and every mesh node within the interface tolerance plus the solver's
    residual bound; after the second, the meshes are within 1e-9 of two oracle steps."""
    import torch

    import paper_1504_00084_gb300 as S
    from gpu_helpers import mesh_tolerance
    from oracle import step as ostep
    probs = oracle_anchor_problems()
    extra = small_mix(W.PREC_FP64, paths=1000, n=1)[0]
    hs = [gpu_problem(p) for p in probs + [extra]]
    stream = torch.cuda.Stream()
    with S.SddBatch(hs, stream=stream) as b:
        b.step()
        stream.synchronize()
        first = [h.mesh() for h in hs[:3]]
        b.step()
        stream.synchronize()
    for prob, h, (g1x, g1y) in zip(probs, hs, first):
        x, y = W.identity_mesh(prob)
        r1 = ostep.step(prob, x, y, prob.t0, 0)
        nodes = r1["nodes"]
        g_est = np.stack([g1x[nodes[:, 1], nodes[:, 0]], g1y[nodes[:, 1], nodes[:, 0]]], 1)
        assert np.abs(g_est - r1["est"]).max() <= 1e-10
        bx, by = ostep.scatter(prob, nodes, r1["est"])
        tol = mesh_tolerance(prob, r1["omega"], bx, by, x, y, 1e-10)
        assert np.abs(g1x - r1["x"]).max() <= tol and np.abs(g1y - r1["y"]).max() <= tol
        r2 = ostep.step(prob, r1["x"], r1["y"], prob.t0 + prob.dt, 1)
        g2x, g2y = h.mesh()
        assert np.abs(g2x - r2["x"]).max() <= 1e-9 and np.abs(g2y - r2["y"]).max() <= 1e-9
        assert h.stats()["step_index"] == 2
    for h in hs:
        h.close()


def test_batch_with_cluster_solved_subdomains_equals_alone():
    """A batch holding a 513 x 513 problem split 2 x 2 (255^2 interior unknowns per subdomain,
    solved by clusters of CTAs) beside small problems: every mesh is bitwise the mesh of stepping
    the problem alone (the small subdomains run the same one-CTA solve in either launch)."""
    import torch

    import paper_1504_00084_gb300 as S
    big = W.c3_mix(64)[0].replace(nx=513, ny=513, px=2, py=2, precision=W.PREC_FP32_KAHAN, paths_per_node=1024,
                                  seed=41)
    probs = [big] + small_mix(W.PREC_FP32_KAHAN, paths=1024, n=3)
    ref = meshes_alone(probs, 1)
    hs = [gpu_problem(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddBatch(hs, stream=stream) as b:
        b.step()
        st = b.stats()
    stream.synchronize()
    assert st["solve_rel_residual"] <= max(p.solve_rtol for p in probs)
    for h, (rx, ry) in zip(hs, ref):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        h.close()
