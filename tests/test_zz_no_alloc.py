"""The allocation-free interface Monte Carlo entry point (sdd_interface_mc_noalloc).

It serves callers that cannot call cudaMalloc (a framework allocator that owns the device
memory budget, or a loop that must not allocate): every intermediate lives in a fixed device
array inside the library.  These tests call it through the C ABI with device buffers and
check it against sdd_interface_mc on the same problem, twice in a row (the shared array keeps
the previous call's contents, so the second call checks that the entry point re-initialises
what it reads), against the CPU oracle, over several path rounds, and that a warm call leaves
the device's free memory unchanged.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # node-estimate tolerance of the other GPU tests (the two paths share kernels)


def smooth_monitor(prob):
    xi = np.arange(prob.nx) / (prob.nx - 1)
    eta = np.arange(prob.ny) / (prob.ny - 1)
    X, Y = np.meshgrid(xi, eta)
    return 1.0 + 3.0 * np.exp(-40 * ((X - 0.4) ** 2 + (Y - 0.55) ** 2))


@pytest.mark.parametrize("precision,periodic,paths", [(W.PREC_FP32_ACC64, 0, 20000), (W.PREC_FP64, 0, 4000),
                                                      (W.PREC_FP32_KAHAN, 1, 20000),
                                                      (W.PREC_FP32_KAHAN, 0, (1 << 19) + 4096)])
def test_noalloc_matches_interface_mc_on_two_calls(precision, periodic, paths):
    """paths = 2^19 + 4096 takes two path rounds (a node runs at most 2^19 paths per round)."""
    import torch

    import paper_1504_00084_gb300 as S
    prob = W.c1_front(precision, periodic=periodic).replace(
        nx=65, ny=65, paths_per_node=paths, monitor_kind=W.MONITOR_NODAL, monitor_params=[])
    x, y = W.sine_mode_mesh(prob, amp=0.01, periodic_mode=bool(periodic))
    om = smooth_monitor(prob)
    params = S.params_from(prob)
    with S.SddProblem(params, x, y) as h:
        h.set_monitor(om)
        est_ref, se_ref, _, _ = h.interface_mc()
    torch.cuda.set_device(0)
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    dom = torch.tensor(om, dtype=torch.float64, device="cuda")
    M = len(est_ref)
    est = torch.empty((M, 2), dtype=torch.float64, device="cuda")
    se = torch.empty((M, 2), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        est.fill_(float("nan"))
        se.fill_(float("nan"))
        st = S.lib.sdd_interface_mc_noalloc(ctypes.byref(params), dx.data_ptr(), dy.data_ptr(),
                                            dom.data_ptr(), 0, est.data_ptr(), se.data_ptr(),
                                            stream.cuda_stream)
        assert st == S.SDD_OK
        torch.cuda.synchronize()
        e, s_ = est.cpu().numpy(), se.cpu().numpy()
        assert np.all(np.isfinite(e)) and np.all(np.isfinite(s_))
        assert np.abs(e - est_ref).max() <= TOL
        assert np.abs(s_ - se_ref).max() <= TOL


def test_noalloc_rejects_what_it_cannot_hold():
    import torch

    import paper_1504_00084_gb300 as S
    prob = W.c1_front(W.PREC_FP32_ACC64).replace(nx=65, ny=65, paths_per_node=20000,
                                                 monitor_kind=W.MONITOR_NODAL)
    x, y = W.identity_mesh(prob)
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dom = torch.ones_like(dx)
    est = torch.empty((10000, 2), dtype=torch.float64, device="cuda")
    se = torch.empty_like(est)
    lib = S.lib

    def call(params, xp=dx.data_ptr()):
        return lib.sdd_interface_mc_noalloc(ctypes.byref(params), xp, dx.data_ptr(), dom.data_ptr(), 0,
                                            est.data_ptr(), se.data_ptr(), None)

    assert call(S.params_from(prob)) == S.SDD_OK
    torch.cuda.synchronize()
    big = S.params_from(prob.replace(nx=1025, ny=1025))        # grid beyond the scratch array
    assert call(big) == S.SDD_ERR_INVALID_ARG
    many = S.params_from(prob.replace(nx=257, ny=257, paths_per_node=1 << 22))  # too many tasks
    assert call(many) == S.SDD_ERR_INVALID_ARG
    adaptive = S.params_from(prob.replace(se_target=1e-3, max_paths_per_node=1 << 20))
    assert call(adaptive) == S.SDD_ERR_INVALID_ARG
    assert call(S.params_from(prob), xp=x.ctypes.data) == S.SDD_ERR_INVALID_ARG  # host pointer


def _device_call(S, prob, x, y, om):
    import torch
    params = S.params_from(prob)
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    dom = torch.tensor(om, dtype=torch.float64, device="cuda")
    return params, dx, dy, dom


def test_noalloc_matches_oracle_and_leaves_free_memory_unchanged():
    """FP64 estimates of the entry point against the CPU oracle (1e-10), on a 33 x 33 grid split
    4 x 2 with a nodal monitor at time-step index 1; and the device's free memory (cudaMemGetInfo) is the
    same before and after a warm call."""
    import torch

    import paper_1504_00084_gb300 as S
    from gpu_helpers import oracle_inputs
    from oracle import mc
    prob = W.c0_small_fp64().replace(px=4, py=2, monitor_kind=W.MONITOR_NODAL, monitor_params=[],
                                     paths_per_node=3000)
    x, y = W.sine_mode_mesh(prob, amp=0.02)
    om = smooth_monitor(prob)
    torch.cuda.set_device(0)
    params, dx, dy, dom = _device_call(S, prob, x, y, om)
    om_o, inp, nodes = oracle_inputs(prob, x, y, prob.t0, 1, om)
    M = len(nodes)
    est = torch.empty((M, 2), dtype=torch.float64, device="cuda")
    se = torch.empty((M, 2), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        return S.lib.sdd_interface_mc_noalloc(ctypes.byref(params), dx.data_ptr(), dy.data_ptr(), dom.data_ptr(),
                                              1, est.data_ptr(), se.data_ptr(), stream.cuda_stream)

    assert call() == S.SDD_OK        # warm: the first call resolves the scratch array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert call() == S.SDD_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    oest, ose, _, _ = mc.interface_mc(prob, x, y, om_o, nodes, 1, np.float64)
    assert np.abs(est.cpu().numpy() - oest).max() <= TOL
    assert np.abs(se.cpu().numpy() - ose).max() <= TOL


def test_noalloc_without_interface_nodes_is_a_no_op():
    import torch

    import paper_1504_00084_gb300 as S
    prob = W.c0_small_fp64().replace(nx=17, ny=17, px=1, py=1, monitor_kind=W.MONITOR_NODAL, monitor_params=[])
    x, y = W.identity_mesh(prob)
    params, dx, dy, dom = _device_call(S, prob, x, y, np.ones_like(x))
    assert S.lib.sdd_interface_mc_noalloc(ctypes.byref(params), dx.data_ptr(), dy.data_ptr(), dom.data_ptr(),
                                          0, None, None, None) == S.SDD_OK
    torch.cuda.synchronize()
