"""The C-ABI library loads, exports every symbol include/sdd.h declares, and its host-only
logic (interface layout, adaptive schedule, argument validation) matches the oracle.
No compute call needs a GPU here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_00084_gb300 as S
    return S


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdd_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(sdd):
    names = declared_functions()
    assert len(names) >= 19
    lib = ctypes.CDLL(sdd.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sdd.EXPORTS)


@pytest.mark.parametrize("nx,ny,px,py,per", [(33, 33, 2, 2, 0), (257, 257, 4, 4, 0), (257, 257, 4, 4, 1),
                                             (65, 129, 8, 2, 0), (9, 9, 1, 1, 0), (9, 9, 1, 1, 1),
                                             (3, 3, 2, 2, 0), (17, 33, 4, 2, 1), (41, 41, 3, 3, 0),
                                             (41, 41, 3, 3, 1), (100, 37, 7, 5, 0), (50, 50, 13, 6, 1)])
def test_interface_layout_matches_oracle(sdd, nx, ny, px, py, per):
    from oracle.layout import interface_nodes
    got = sdd.sdd_interface_layout(nx, ny, px, py, per)
    want = interface_nodes(nx, ny, px, py, per)
    assert np.array_equal(got, want)


def test_adaptive_schedule_matches_oracle(sdd):
    from oracle.mc import next_total
    rng = np.random.default_rng(0)
    cases = [(4096, 1e-4, 1e-4, 10 ** 7), (4096, 2e-4, 1e-4, 10 ** 7), (4096, 1.01e-4, 1e-4, 10 ** 7),
             (4096, 1.0, 1e-4, 50000), (50000, 1.0, 1e-4, 50000), (1000, 0.0, 1e-4, 10 ** 6)]
    for _ in range(500):
        n = int(rng.integers(2, 10 ** 7))
        t = float(10 ** rng.uniform(-6, -2))
        cases.append((n, float(t * 10 ** rng.uniform(-1, 2)), t, int(n + rng.integers(0, 10 ** 8))))
    for n, se, t, mx in cases:
        assert sdd.sdd_adaptive_next_total(n, se, t, mx) == next_total(n, se, t, mx), (n, se, t, mx)


def base_params(sdd, **kw):
    import workloads as W
    return sdd.params_from(W.c0_small_fp64(), **kw)


@pytest.mark.parametrize("field,value", [("nx", 2), ("px", 40), ("py", 0), ("substeps", 0),
                                         ("paths_per_node", 1), ("iface_stride", -1), ("tau", 0.0),
                                         ("precision", 7), ("form", 2), ("solve_rtol", 0.0),
                                         ("periodic", 2), ("se_target", -1.0),
                                         ("moving_boundary", 2), ("subdomain_scheme", 3),
                                         ("fe_max_substeps", -1)])
def test_invalid_params_rejected_before_any_device_work(sdd, field, value):
    import workloads as W
    p = base_params(sdd)
    setattr(p, field, value)
    x, y = W.identity_mesh(W.c0_small_fp64())
    h = ctypes.c_void_p()
    st = sdd.lib.sdd_create_problem(ctypes.byref(p), x.ctypes.data, y.ctypes.data, None, ctypes.byref(h))
    assert st == sdd.SDD_ERR_INVALID_ARG
    assert h.value is None
    assert len(sdd.lib.sdd_last_error()) > 0


def test_adaptive_cap_validated(sdd):
    import workloads as W
    p = base_params(sdd, se_target=1e-3, max_paths_per_node=10)
    x, y = W.identity_mesh(W.c0_small_fp64())
    h = ctypes.c_void_p()
    assert sdd.lib.sdd_create_problem(ctypes.byref(p), x.ctypes.data, y.ctypes.data, None,
                                      ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG


def test_status_strings(sdd):
    for s in range(7):
        assert len(sdd.lib.sdd_status_string(s)) > 0


def test_checkpoint_load_rejects_bad_files_before_device_work(sdd, tmp_path):
    h = ctypes.c_void_p()
    missing = str(tmp_path / "none.ckpt").encode()
    assert sdd.lib.sdd_load(missing, None, ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(100))
    assert sdd.lib.sdd_load(str(bad).encode(), None, ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG
    # right magic and record size, parameters that fail validation
    p = sdd.SddParams()
    body = b"SDDCKPT1" + ctypes.sizeof(p).to_bytes(4, "little") + bytes(p)
    short = tmp_path / "short.ckpt"
    short.write_bytes(body + bytes(8))
    assert sdd.lib.sdd_load(str(short).encode(), None, ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG
    assert sdd.lib.sdd_save(None, str(short).encode()) == sdd.SDD_ERR_INVALID_ARG



@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("shape", [(33, 33, 4, 4), (41, 25, 5, 3), (65, 65, 8, 2), (9, 17, 1, 2), (41, 41, 3, 3),
                                   (50, 37, 7, 4)])
@pytest.mark.parametrize("stride", [0, 1, 2, 3, 4, 7, 40])
def test_interface_sampling_matches_oracle(sdd, periodic, shape, stride):
    from oracle.layout import interface_sampling
    nx, ny, px, py = shape
    p = base_params(sdd, nx=nx, ny=ny, px=px, py=py, periodic=periodic, iface_stride=stride)
    got = sdd.sdd_interface_sampling(p)
    want, _ = interface_sampling(nx, ny, px, py, periodic, stride)
    assert np.array_equal(got, want)



def test_moving_boundary_needs_a_dirichlet_domain(sdd):
    p = base_params(sdd, periodic=1, moving_boundary=1)
    x = np.zeros((p.ny, p.nx))
    h = ctypes.c_void_p()
    assert sdd.lib.sdd_create_problem(ctypes.byref(p), x.ctypes.data, x.ctypes.data, None,
                                      ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG


def test_interface_node_limit(sdd):
    """A round's tasks are counted in 32 bits: problems (and server pools) with 2^23 or more
    interface nodes are rejected before any device work.  4097^2 split 4096 x 4096 has 4095^2."""
    p = base_params(sdd, nx=4097, ny=4097, px=4096, py=4096)
    x = np.zeros((4097, 4097))
    h = ctypes.c_void_p()
    assert sdd.lib.sdd_create_problem(ctypes.byref(p), x.ctypes.data, x.ctypes.data, None,
                                      ctypes.byref(h)) == sdd.SDD_ERR_INVALID_ARG
    assert b"2^23" in sdd.lib.sdd_last_error()


def test_noalloc_source_calls_no_allocator():
    """The allocation-free entry point's translation unit names no device or host allocation
    routine of the CUDA runtime or driver (its intermediates live in a fixed device array)."""
    import re
    src = open(os.path.join(ROOT, "paper_1504_00084_gb300", "csrc", "sdd_noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", src)   # comments may name what the code avoids
    for name in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaFreeAsync", "cudaHostAlloc", "cudaMallocHost",
                 "cudaMallocManaged", "cudaMallocPitch", "cudaMalloc3D", "cudaMallocArray", "cuMemAlloc",
                 "cuMemCreate", "cudaMemPool", "malloc(", "new ", "std::vector"):
        assert name not in code, name
