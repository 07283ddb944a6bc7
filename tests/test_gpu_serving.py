"""Serving with continuous batching (sdd_server_*): every request's new mesh and interface
estimates are bitwise those of stepping the same problem alone, whether it ran alone, joined
a running set mid-flight, waited in the queue for memory, or reused the device state of an
earlier request; admission, budget and rejection rules."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_problem
from test_gpu_batch import small_mix

pytestmark = pytest.mark.gpu


def server_params(precision, paths, se_target=0.0, max_paths=0, max_resident=64, max_nodes=1 << 16,
                  budget=0, round_paths=0):
    import paper_1504_00084_gb300 as S
    q = S.SddServerParams()
    q.precision = precision
    q.max_resident = max_resident
    q.max_nodes = max_nodes
    q.mem_budget_bytes = budget
    q.se_target = se_target
    q.paths_per_node = paths
    q.max_paths_per_node = max_paths if se_target > 0 else paths
    q.round_paths = round_paths
    return q


def alone(prob, steps=1):
    """Mesh after `steps` alone steps and the interface estimates of the last step."""
    h = gpu_problem(prob)
    for _ in range(steps - 1):
        h.step()
    est, se, _, _ = h.interface_mc()
    h2 = gpu_problem(prob)
    for _ in range(steps):
        h2.step()
    x, y = h2.mesh()
    h.close()
    h2.close()
    return x, y, est, se


def submit(srv, prob, x=None, y=None, step_index=0):
    import paper_1504_00084_gb300 as S
    if x is None:
        x, y = W.identity_mesh(prob)
    kind = prob.monitor_kind
    mp = None if kind == W.MONITOR_NODAL else np.asarray(prob.monitor_params, dtype=np.float64)
    return srv.submit(S.params_from(prob), np.ascontiguousarray(x), np.ascontiguousarray(y), kind, mp,
                      step_index=step_index)


def drain(srv, expect, max_calls=100000):
    done = []
    for _ in range(max_calls):
        srv.progress()
        done += srv.poll()
        if len(done) >= expect:
            return done
    raise AssertionError("server did not complete its requests")


def mixed_requests(precision, paths, se_target):
    probs = small_mix(precision, paths=paths, se_target=se_target)
    # one subdomain: no interface node, the request is a plain single-domain solve
    probs.append(probs[0].replace(px=1, py=1, seed=99))
    return probs


@pytest.mark.parametrize("precision,round_paths", [(W.PREC_FP32_KAHAN, 0), (W.PREC_FP64, 0),
                                                   (W.PREC_FP32_KAHAN, 100000)])
def test_server_results_bitwise_equal_problems_alone(precision, round_paths):
    """round_paths > 0: rounds hold ~50 tasks, so most rounds run only the oldest requests'
    nodes and leave the others' chunks for later rounds."""
    import torch

    import paper_1504_00084_gb300 as S
    se_target = 6e-3 if precision != W.PREC_FP64 else 1.2e-2
    probs = mixed_requests(precision, 2048, se_target)
    refs = [alone(p) for p in probs]
    stream = torch.cuda.Stream()
    with S.SddServer(server_params(precision, 2048, se_target, 1 << 16, round_paths=round_paths),
                     stream) as srv:
        ids = [submit(srv, p) for p in probs[:3]]
        srv.progress()
        srv.progress()
        ids += [submit(srv, p) for p in probs[3:]]  # join a running set
        done = drain(srv, len(ids))
        assert sorted(done) == sorted(ids)
        for rid, prob, (rx, ry, rest, rse) in zip(ids, probs, refs):
            out = srv.result(rid)
            assert out["status"] == S.SDD_OK
            assert np.array_equal(out["x"], rx) and np.array_equal(out["y"], ry)
            assert np.array_equal(out["est"], rest) and np.array_equal(out["se"], rse)
            st = out["stats"]
            assert st["step_index"] == 1 and st["nodes_not_reached"] == 0
            assert st["max_se"] <= se_target
        s = srv.stats()
        assert s["completed"] == s["collected"] == len(probs)
        assert s["rounds"] >= 2 and s["mc_kernel_ms"] > 0


def test_server_fixed_paths_and_later_step_index():
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=4096, n=4)
    stream = torch.cuda.Stream()
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 4096), stream) as srv:
        for prob in probs:
            # the mesh after one alone step, advanced by the server as step index 1
            h = gpu_problem(prob)
            h.step()
            x1, y1 = h.mesh()
            h.step()
            x2, y2 = h.mesh()
            h.close()
            rid = submit(srv, prob, x1, y1, step_index=1)
            drain(srv, 1)
            out = srv.result(rid)
            assert np.array_equal(out["x"], x2) and np.array_equal(out["y"], y2)
            assert out["stats"]["step_index"] == 2
            assert out["stats"]["paths"] == 4096 * out["stats"]["M"]


def test_server_budget_queueing_pool_reuse_and_cache():
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=6, se_target=6e-3)
    small = [p.replace(nx=33, ny=33, px=4, py=4, periodic=0, seed=200 + k) for k, p in enumerate(probs)]
    big = small[0].replace(nx=65, ny=65, px=2, py=2, seed=300)
    refs = [alone(p) for p in small]
    stream = torch.cuda.Stream()
    # bytes of one 33x33 request's state
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, 6e-3, 1 << 16), stream) as srv:
        rid = submit(srv, small[0])
        drain(srv, 1)
        one = srv.stats()["resident_bytes"]
        srv.result(rid)
    assert one > 0
    M33 = 3 * 31 * 2 - 9
    # room for two requests' state and two requests' nodes: the rest queue, ranges and state recycle
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, 6e-3, 1 << 16, max_resident=3,
                                   max_nodes=2 * M33, budget=2 * one + one // 2), stream) as srv:
        ids = [submit(srv, p) for p in small]
        bad = submit(srv, big)  # more state than the whole budget: completes with SDD_ERR_OOM
        got = {}
        for _ in range(100000):
            srv.progress()
            st = srv.stats()
            assert st["running"] + st["finishing"] + st["done"] <= 3
            assert st["resident_bytes"] <= 2 * one + one // 2
            for rid in srv.poll():
                if rid == bad:
                    with pytest.raises(S.SddError) as e:
                        srv.result(rid)
                    assert e.value.status == S.SDD_ERR_OOM
                    got[rid] = None
                else:
                    got[rid] = srv.result(rid)
            if len(got) == len(ids) + 1:
                break
        for rid, (rx, ry, rest, _) in zip(ids, refs):
            assert np.array_equal(got[rid]["x"], rx) and np.array_equal(got[rid]["y"], ry)
            assert np.array_equal(got[rid]["est"], rest)
        st = srv.stats()
        assert st["allocations"] <= 2  # later requests reuse collected state of the same shape
        assert st["pool_high_water"] <= 2 * M33


def test_server_rejections():
    import torch

    import paper_1504_00084_gb300 as S
    prob = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=1)[0]
    stream = torch.cuda.Stream()
    with pytest.raises(S.SddError):
        S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, max_resident=0), stream)
    with pytest.raises(S.SddError):
        S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048), None)
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, max_nodes=10), stream) as srv:
        x, y = W.identity_mesh(prob)
        with pytest.raises(S.SddError):  # precision differs from the server's
            srv.submit(S.params_from(prob.replace(precision=W.PREC_FP64)), x, y)
        with pytest.raises(S.SddError):  # more interface nodes than the pool
            srv.submit(S.params_from(prob), x, y)
        small = prob.replace(nx=9, ny=9, px=2, py=1, periodic=0)
        xs, ys = W.identity_mesh(small)
        xb = xs.copy()
        xb[0, 3] += 0.01
        with pytest.raises(S.SddError):  # Dirichlet boundary moved
            srv.submit(S.params_from(small), xb, ys)
        with pytest.raises(S.SddError):  # unknown id
            S.sdd_server_result(srv.h, 12345)
        rid = srv.submit(S.params_from(small), xs, ys)
        with pytest.raises(S.SddError):  # not completed yet
            S.sdd_server_result(srv.h, rid)
        drain(srv, 1)
        out = srv.result(rid)
        h = S.SddProblem(S.params_from(small), xs, ys)
        h.step()
        rx, ry = h.mesh()
        h.close()
        assert np.array_equal(out["x"], rx) and np.array_equal(out["y"], ry)


def test_server_cancellation():
    """A cancelled queued request completes at once, a cancelled running one leaves the plan at
    the next round; both report SDD_ERR_CANCELLED, and the other requests are unaffected."""
    import torch

    import paper_1504_00084_gb300 as S
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=5, se_target=6e-3)
    refs = {k: alone(probs[k]) for k in (0, 2, 4)}
    stream = torch.cuda.Stream()
    with S.SddServer(server_params(W.PREC_FP32_KAHAN, 2048, 6e-3, 1 << 16, max_resident=2), stream) as srv:
        ids = [submit(srv, p) for p in probs]
        srv.progress()                      # admits the first two and launches a round
        assert srv.stats()["running"] == 2 and srv.stats()["queued"] == 3
        srv.cancel(ids[1])                  # running
        srv.cancel(ids[3])                  # queued
        with pytest.raises(S.SddError):
            srv.cancel(987654)
        got = {}
        for _ in range(100000):
            srv.progress()
            for rid in srv.poll():
                k = ids.index(rid)
                if k in (1, 3):
                    with pytest.raises(S.SddError) as e:
                        srv.result(rid)
                    assert e.value.status == S.SDD_ERR_CANCELLED
                    got[k] = None
                else:
                    got[k] = srv.result(rid)
            if len(got) == 5:
                break
        assert len(got) == 5
        for k, (rx, ry, rest, _) in refs.items():
            assert np.array_equal(got[k]["x"], rx) and np.array_equal(got[k]["y"], ry)
            assert np.array_equal(got[k]["est"], rest)


def test_served_fp64_requests_match_oracle():
    """Served requests against the oracle itself: the three FP64 problems of uneven shapes of the
    batch anchor test, served at an adaptive SE target (two submitted first, one joining the
    running set).  Each request's interface estimates are the oracle's within 1e-10 with the
    oracle's adaptive path counts, and its new mesh is the oracle's within the interface
    tolerance plus the solver's residual bound."""
    import torch

    import paper_1504_00084_gb300 as S
    from gpu_helpers import mesh_tolerance
    from oracle import step as ostep
    from test_gpu_batch import oracle_anchor_problems
    se_target = 1.2e-2
    probs = [p.replace(paths_per_node=2048, se_target=se_target, max_paths_per_node=1 << 16)
             for p in oracle_anchor_problems()]
    stream = torch.cuda.Stream()
    with S.SddServer(server_params(W.PREC_FP64, 2048, se_target, 1 << 16), stream) as srv:
        ids = [submit(srv, p) for p in probs[:2]]
        srv.progress()
        ids.append(submit(srv, probs[2]))
        drain(srv, len(ids))
        outs = [srv.result(rid) for rid in ids]
    for prob, out in zip(probs, outs):
        assert out["status"] == S.SDD_OK
        x, y = W.identity_mesh(prob)
        r = ostep.step(prob, x, y, prob.t0, 0)
        assert np.abs(out["est"] - r["est"]).max() <= 1e-10
        assert np.abs(out["se"] - r["se"]).max() <= 1e-10
        assert out["stats"]["paths"] == int(r["n_used"].sum())
        bx, by = ostep.scatter(prob, r["nodes"], r["est"])
        tol = mesh_tolerance(prob, r["omega"], bx, by, x, y, 1e-10)
        assert np.abs(out["x"] - r["x"]).max() <= tol and np.abs(out["y"] - r["y"]).max() <= tol
