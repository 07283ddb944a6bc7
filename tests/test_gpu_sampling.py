"""Interface sampling (iface_stride > 1, Sec. 3.6): Monte Carlo at a sample of the interface
nodes, linear interpolation along the interface lines elsewhere.  Sampled nodes keep their node
ids, so their estimates are bitwise those of the full evaluation; interpolated nodes are bitwise
the oracle's interpolation of the GPU's sampled estimates; the whole step matches the oracle's
step with the same sampling; batches and the server give the same results as a problem alone."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem
from oracle import step as ostep
from oracle.layout import interface_sampling
from gpu_helpers import mesh_tolerance

pytestmark = pytest.mark.gpu


def case(periodic, precision, stride):
    prob = W.c0_small_fp64().replace(precision=precision, paths_per_node=1000 if precision == W.PREC_FP64 else 4096,
                                     iface_stride=stride)
    if periodic:
        prob = prob.replace(periodic=1, monitor_params=[6.0, 40.0, 0.3, 0.6])
    return prob


@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32_KAHAN])
@pytest.mark.parametrize("stride", [2, 3, 5])
def test_sampled_nodes_equal_full_and_interpolation_matches_oracle(periodic, precision, stride):
    import paper_1504_00084_gb300 as S
    full = case(periodic, precision, 0)
    samp = case(periodic, precision, stride)
    h1 = gpu_problem(full)
    e1, s1, n1, _ = h1.interface_mc()
    h2 = gpu_problem(samp)
    e2, s2, n2, _ = h2.interface_mc()
    mask = S.sdd_interface_sampling(S.params_from(samp))
    want_mask, fill = interface_sampling(samp.nx, samp.ny, samp.px, samp.py, samp.periodic, stride, samp.Lx, samp.Ly)
    assert np.array_equal(mask, want_mask) and 0 < mask.sum() < len(mask)
    assert np.array_equal(e2[mask], e1[mask]) and np.array_equal(s2[mask], s1[mask])
    assert np.array_equal(n2[mask], n1[mask]) and np.all(n2[~mask] == 0) and np.all(s2[~mask] == 0)
    blank = e2.copy()
    blank[~mask] = np.nan
    assert np.array_equal(fill(blank), e2)
    st = h2.stats()
    assert st["paths"] == n2.sum()
    h1.close()
    h2.close()


@pytest.mark.parametrize("periodic", [0, 1])
def test_full_step_with_sampling_fp64(periodic):
    prob = case(periodic, W.PREC_FP64, 3)
    x, y = W.identity_mesh(prob)
    h = gpu_problem(prob, x, y)
    gx, gy, _ = h.step()
    r = ostep.step(prob, x, y, prob.t0, 0)
    bx, by = ostep.scatter(prob, r["nodes"], r["est"])
    tol = mesh_tolerance(prob, r["omega"], bx, by, x, y, 1e-10)
    assert np.abs(gx - r["x"]).max() <= tol and np.abs(gy - r["y"]).max() <= tol
    h.close()


def test_sampling_in_batches_and_server_equals_alone():
    import torch

    import paper_1504_00084_gb300 as S
    from test_gpu_batch import small_mix
    from test_gpu_serving import alone, drain, server_params, submit
    probs = [p.replace(iface_stride=s) for p, s in zip(small_mix(W.PREC_FP32_KAHAN, paths=2048, n=4, se_target=6e-3),
                                                         [3, 0, 2, 4])]
    refs = [alone(p) for p in probs]
    hs = [gpu_problem(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddBatch(hs, stream=stream) as b:
        b.step()
        b.stats()
    for h, (rx, ry, _, _) in zip(hs, refs):
        gx, gy = h.mesh()
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
        h.close()
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, 6e-3, 1 << 16), stream) as srv:
        ids = [submit(srv, p) for p in probs]
        drain(srv, len(ids))
        for rid, (rx, ry, rest, _) in zip(ids, refs):
            out = srv.result(rid)
            assert np.array_equal(out["x"], rx) and np.array_equal(out["y"], ry)
            assert np.array_equal(out["est"], rest)
