"""The allocation-free interface Monte Carlo entry point (sdd_interface_mc_noalloc).

It serves callers that cannot call cudaMalloc (a framework allocator that owns the device
memory budget, or a loop that must not allocate): every intermediate lives in a fixed device
array inside the library.  These tests call it through the C ABI with device buffers and
check it against sdd_interface_mc on the same problem, twice in a row (the shared array keeps
the previous call's contents, so the second call checks that the entry point re-initialises
what it reads).  Collected last on purpose."""
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


@pytest.mark.parametrize("precision,periodic", [(W.PREC_FP32_ACC64, 0), (W.PREC_FP64, 0),
                                                (W.PREC_FP32_KAHAN, 1)])
def test_noalloc_matches_interface_mc_on_two_calls(precision, periodic):
    import torch

    import paper_1504_00084_gb300 as S
    prob = W.c1_front(precision, periodic=periodic).replace(
        nx=65, ny=65, paths_per_node=20000 if precision != W.PREC_FP64 else 4000,
        monitor_kind=W.MONITOR_NODAL, monitor_params=[])
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
