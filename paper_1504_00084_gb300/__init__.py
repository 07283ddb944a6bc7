"""Python binding of the GB300 SDD mesh-generator library (argument marshalling only).

Every function here forwards to the C ABI of include/sdd.h in the in-tree CUDA library
paper_1504_00084_gb300/_build/libsdd.so; every step of the method runs in its kernels.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); torch supplies device
memory and streams only.  There is no CPU fallback: importing this module fails loudly if
the CUDA library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SDD_LIB_PATH selects another build of the same library (e.g. the bounds-checked one).
LIB_PATH = os.environ.get("SDD_LIB_PATH") or os.path.join(_HERE, "_build", "libsdd.so")

SDD_OK = 0
SDD_ERR_INVALID_ARG = 1
SDD_ERR_OOM = 2
SDD_ERR_CUDA = 3
SDD_ERR_NOT_CONVERGED = 4
SDD_ERR_SE_NOT_REACHED = 5
SDD_ERR_NO_DEVICE = 6
SDD_ERR_CANCELLED = 7

SDD_FORM_DIV, SDD_FORM_WINSLOW = 0, 1
SDD_FP64, SDD_FP32_ACC64, SDD_FP32_KAHAN = 0, 1, 2
SDD_MONITOR_NODAL, SDD_MONITOR_GAUSS, SDD_MONITOR_FRONT, SDD_MONITOR_BUMPS, SDD_MONITOR_RINGS = 0, 1, 2, 3, 4


class SddParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("px", ctypes.c_int32),
                ("py", ctypes.c_int32), ("periodic", ctypes.c_int32), ("form", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("bicubic", ctypes.c_int32), ("bb_test", ctypes.c_int32),
                ("substeps", ctypes.c_int32), ("solve_max_iter", ctypes.c_int32),
                ("iface_stride", ctypes.c_int32), ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("tau", ctypes.c_double), ("dt", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("paths_per_node", ctypes.c_int64), ("max_paths_per_node", ctypes.c_int64),
                ("se_target", ctypes.c_double), ("solve_rtol", ctypes.c_double), ("t0", ctypes.c_double),
                ("subdomain_scheme", ctypes.c_int32), ("fe_max_substeps", ctypes.c_int32),
                ("moving_boundary", ctypes.c_int32)]


class SddStats(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("step_index", ctypes.c_int32), ("t", ctypes.c_double),
                ("path_steps", ctypes.c_int64), ("paths", ctypes.c_int64), ("mc_rounds", ctypes.c_int32),
                ("nodes_not_reached", ctypes.c_int32), ("max_se", ctypes.c_double),
                ("solve_iters_max", ctypes.c_int32), ("solve_outer_max", ctypes.c_int32),
                ("solve_rel_residual", ctypes.c_double), ("mc_kernel_ms", ctypes.c_double),
                ("mc_kernel_launches", ctypes.c_int32), ("reserved1", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("solve_kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SddMcConfig(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("paths_per_task", ctypes.c_int32), ("max_blocks_per_sm", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SddServerParams(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_resident", ctypes.c_int32),
                ("max_nodes", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_int64),
                ("se_target", ctypes.c_double), ("paths_per_node", ctypes.c_int64),
                ("max_paths_per_node", ctypes.c_int64), ("round_paths", ctypes.c_int64)]


class SddServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("collected", ctypes.c_int64),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("finishing", ctypes.c_int32),
                ("done", ctypes.c_int32), ("rounds", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("mc_kernel_ms", ctypes.c_double), ("path_steps", ctypes.c_int64),
                ("interface_nodes", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("cached_bytes", ctypes.c_int64), ("pool_bytes", ctypes.c_int64),
                ("pool_high_water", ctypes.c_int64), ("allocations", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "sdd_create_problem", "sdd_destroy_problem", "sdd_set_stream", "sdd_set_mesh", "sdd_get_mesh",
    "sdd_set_monitor", "sdd_set_monitor_analytic", "sdd_interface_mc", "sdd_subdomain_solve",
    "sdd_step", "sdd_get_stats", "sdd_get_interface_nodes", "sdd_interface_layout",
    "sdd_adaptive_next_total", "sdd_get_monitor", "sdd_debug_paths", "sdd_debug_philox",
    "sdd_debug_unit_math", "sdd_interface_mc_range", "sdd_step_from_interface",
    "sdd_status_string", "sdd_last_error", "sdd_interface_mc_noalloc",
    "sdd_batch_create", "sdd_batch_step", "sdd_batch_get_stats", "sdd_batch_destroy", "sdd_batch_tune",
    "sdd_mesh_quality",
    "sdd_server_create", "sdd_server_submit", "sdd_server_progress", "sdd_server_poll",
    "sdd_server_result", "sdd_server_get_stats", "sdd_server_destroy",
    "sdd_save", "sdd_load", "sdd_interface_sampling", "sdd_step_mkp", "sdd_server_cancel",
    "sdd_debug_bounds_violations", "sdd_get_mc_config", "sdd_set_mc_config", "sdd_tune",
    "sdd_batch_get_mc_config", "sdd_batch_set_mc_config", "sdd_batch_tune_mc",
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sdd_create_problem": ([ctypes.POINTER(SddParams), P, P, P, ctypes.POINTER(P)], I32),
        "sdd_destroy_problem": ([P], None),
        "sdd_set_stream": ([P, P], I32),
        "sdd_set_mesh": ([P, P, P], I32),
        "sdd_get_mesh": ([P, P, P], I32),
        "sdd_set_monitor": ([P, P], I32),
        "sdd_set_monitor_analytic": ([P, I32, P, I32], I32),
        "sdd_interface_mc": ([P, P, P, P], I32),
        "sdd_subdomain_solve": ([P, P, P, P], I32),
        "sdd_step": ([P, P, P], I32),
        "sdd_get_stats": ([P, ctypes.POINTER(SddStats)], I32),
        "sdd_get_interface_nodes": ([P, P, ctypes.POINTER(I32)], I32),
        "sdd_interface_layout": ([I32, I32, I32, I32, I32, P, ctypes.POINTER(I32)], I32),
        "sdd_adaptive_next_total": ([I64, F64, F64, I64], I64),
        "sdd_get_monitor": ([P, P, P, P], I32),
        "sdd_debug_paths": ([P, I32, I64, I64, P, P, P], I32),
        "sdd_debug_philox": ([P, P, I64, P], I32),
        "sdd_debug_unit_math": ([P, I64, P], I32),
        "sdd_interface_mc_range": ([P, I32, I32, P, P, P], I32),
        "sdd_step_from_interface": ([P, P, P, P], I32),
        "sdd_debug_bounds_violations": ([], I64),
        "sdd_interface_mc_noalloc": ([ctypes.POINTER(SddParams), P, P, P, I32, P, P, P], I32),
        "sdd_batch_create": ([P, I32, P, I32, ctypes.POINTER(P)], I32),
        "sdd_batch_step": ([P], I32),
        "sdd_batch_tune": ([P, I32, ctypes.POINTER(I32)], I32),
        "sdd_batch_get_stats": ([P, ctypes.POINTER(SddStats)], I32),
        "sdd_get_mc_config": ([P, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_set_mc_config": ([P, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_tune": ([P, I32, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_batch_get_mc_config": ([P, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_batch_set_mc_config": ([P, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_batch_tune_mc": ([P, I32, ctypes.POINTER(SddMcConfig)], I32),
        "sdd_batch_destroy": ([P], None),
        "sdd_mesh_quality": ([P, P, ctypes.POINTER(F64), ctypes.POINTER(F64)], I32),
        "sdd_server_create": ([ctypes.POINTER(SddServerParams), P, ctypes.POINTER(P)], I32),
        "sdd_server_submit": ([P, ctypes.POINTER(SddParams), P, P, I32, P, I32, P, I32,
                               ctypes.POINTER(I64)], I32),
        "sdd_server_progress": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32)], I32),
        "sdd_server_poll": ([P, P, I32, ctypes.POINTER(I32)], I32),
        "sdd_server_result": ([P, I64, P, P, P, P, ctypes.POINTER(SddStats)], I32),
        "sdd_server_get_stats": ([P, ctypes.POINTER(SddServerStats)], I32),
        "sdd_server_destroy": ([P], None),
        "sdd_server_cancel": ([P, I64], I32),
        "sdd_save": ([P, ctypes.c_char_p], I32),
        "sdd_step_mkp": ([P, I32, P, P], I32),
        "sdd_interface_sampling": ([ctypes.POINTER(SddParams), P, ctypes.POINTER(I32)], I32),
        "sdd_load": ([ctypes.c_char_p, P, ctypes.POINTER(P)], I32),
        "sdd_status_string": ([I32], ctypes.c_char_p),
        "sdd_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


class SddError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.sdd_status_string(status).decode()
        detail = lib.sdd_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def _check(status: int, where: str, ok=(SDD_OK,)):
    if status not in ok:
        raise SddError(status, where)
    return status


def _ptr(a) -> Optional[int]:
    """Raw address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def params_from(prob, **overrides) -> SddParams:
    """sdd_params from a workloads.Problem-like object (attributes of the same names)."""
    p = SddParams()
    for name, _ in SddParams._fields_:
        if hasattr(prob, name):
            setattr(p, name, getattr(prob, name))
    if getattr(prob, "max_paths_per_node", 0) <= 0:
        p.max_paths_per_node = p.paths_per_node
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


# --------------------------------------------------------------------------------------
# Same-name wrappers of the C ABI.
# --------------------------------------------------------------------------------------

def sdd_create_problem(params: SddParams, x0, y0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib.sdd_create_problem(ctypes.byref(params), _ptr(x0), _ptr(y0), _stream_handle(stream),
                                  ctypes.byref(h)), "sdd_create_problem")
    return h.value


def sdd_destroy_problem(h: int) -> None:
    lib.sdd_destroy_problem(h)


def sdd_set_stream(h: int, stream) -> None:
    _check(lib.sdd_set_stream(h, _stream_handle(stream)), "sdd_set_stream")


def sdd_set_mesh(h: int, x, y) -> None:
    _check(lib.sdd_set_mesh(h, _ptr(x), _ptr(y)), "sdd_set_mesh")


def sdd_get_mesh(h: int, x, y) -> None:
    _check(lib.sdd_get_mesh(h, _ptr(x), _ptr(y)), "sdd_get_mesh")


def sdd_set_monitor(h: int, omega) -> None:
    _check(lib.sdd_set_monitor(h, _ptr(omega)), "sdd_set_monitor")


def sdd_set_monitor_analytic(h: int, kind: int, params) -> None:
    arr = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib.sdd_set_monitor_analytic(h, kind, arr.ctypes.data if arr.size else None, arr.size),
           "sdd_set_monitor_analytic")


def sdd_interface_mc(h: int, est_xy=None, se_xy=None, paths_used=None, allow_se_not_reached=True) -> int:
    ok = (SDD_OK, SDD_ERR_SE_NOT_REACHED) if allow_se_not_reached else (SDD_OK,)
    return _check(lib.sdd_interface_mc(h, _ptr(est_xy), _ptr(se_xy), _ptr(paths_used)),
                  "sdd_interface_mc", ok)


def sdd_interface_mc_range(h: int, node_begin: int, node_end: int, est_xy=None, se_xy=None, paths_used=None,
                           allow_se_not_reached=True) -> int:
    ok = (SDD_OK, SDD_ERR_SE_NOT_REACHED) if allow_se_not_reached else (SDD_OK,)
    return _check(lib.sdd_interface_mc_range(h, node_begin, node_end, _ptr(est_xy), _ptr(se_xy), _ptr(paths_used)),
                  "sdd_interface_mc_range", ok)


def sdd_step_from_interface(h: int, iface_xy, x_out=None, y_out=None) -> int:
    return _check(lib.sdd_step_from_interface(h, _ptr(iface_xy), _ptr(x_out), _ptr(y_out)),
                  "sdd_step_from_interface")


def sdd_subdomain_solve(h: int, iface_xy=None, x_out=None, y_out=None) -> int:
    return _check(lib.sdd_subdomain_solve(h, _ptr(iface_xy), _ptr(x_out), _ptr(y_out)), "sdd_subdomain_solve")


def sdd_step(h: int, x_out=None, y_out=None, allow_se_not_reached=True) -> int:
    ok = (SDD_OK, SDD_ERR_SE_NOT_REACHED) if allow_se_not_reached else (SDD_OK,)
    return _check(lib.sdd_step(h, _ptr(x_out), _ptr(y_out)), "sdd_step", ok)


def sdd_step_mkp(h: int, K: int, x_out=None, y_out=None, allow_se_not_reached=True) -> int:
    ok = (SDD_OK, SDD_ERR_NOT_CONVERGED) + ((SDD_ERR_SE_NOT_REACHED,) if allow_se_not_reached else ())
    return _check(lib.sdd_step_mkp(h, K, _ptr(x_out), _ptr(y_out)), "sdd_step_mkp", ok=ok)


def sdd_get_stats(h: int) -> dict:
    s = SddStats()
    _check(lib.sdd_get_stats(h, ctypes.byref(s)), "sdd_get_stats")
    return s.as_dict()


def sdd_get_interface_nodes(h: int) -> np.ndarray:
    M = ctypes.c_int32()
    _check(lib.sdd_get_interface_nodes(h, None, ctypes.byref(M)), "sdd_get_interface_nodes")
    ij = np.zeros((M.value, 2), dtype=np.int32)
    _check(lib.sdd_get_interface_nodes(h, ij.ctypes.data if M.value else None, ctypes.byref(M)),
           "sdd_get_interface_nodes")
    return ij


def sdd_interface_layout(nx: int, ny: int, px: int, py: int, periodic: int) -> np.ndarray:
    M = ctypes.c_int32()
    _check(lib.sdd_interface_layout(nx, ny, px, py, periodic, None, ctypes.byref(M)), "sdd_interface_layout")
    ij = np.zeros((M.value, 2), dtype=np.int32)
    if M.value:
        _check(lib.sdd_interface_layout(nx, ny, px, py, periodic, ij.ctypes.data, ctypes.byref(M)),
               "sdd_interface_layout")
    return ij


def sdd_interface_sampling(params: SddParams) -> np.ndarray:
    """bool array over the interface nodes: True where Monte Carlo runs (params.iface_stride)."""
    M = ctypes.c_int32()
    _check(lib.sdd_interface_sampling(ctypes.byref(params), None, ctypes.byref(M)), "sdd_interface_sampling")
    out = np.zeros(max(M.value, 1), dtype=np.int32)
    _check(lib.sdd_interface_sampling(ctypes.byref(params), out.ctypes.data, ctypes.byref(M)),
           "sdd_interface_sampling")
    return out[:M.value].astype(bool)


def sdd_adaptive_next_total(n_done: int, se: float, target: float, max_paths: int) -> int:
    return int(lib.sdd_adaptive_next_total(n_done, se, target, max_paths))


def sdd_get_monitor(h: int, omega=None, w_xi=None, w_eta=None) -> None:
    _check(lib.sdd_get_monitor(h, _ptr(omega), _ptr(w_xi), _ptr(w_eta)), "sdd_get_monitor")


def sdd_debug_paths(h: int, node: int, p_begin: int, n_paths: int):
    val = np.zeros((n_paths, 2), dtype=np.float64)
    steps = np.zeros(n_paths, dtype=np.int32)
    side = np.zeros(n_paths, dtype=np.int8)
    _check(lib.sdd_debug_paths(h, node, p_begin, n_paths, val.ctypes.data, steps.ctypes.data,
                               side.ctypes.data), "sdd_debug_paths")
    return val, steps, side


def sdd_debug_bounds_violations() -> int:
    """Out-of-range gather indices met so far (bounds-checked build), -1 in a normal build."""
    return int(lib.sdd_debug_bounds_violations())


def sdd_debug_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(lib.sdd_debug_philox(ctr.ctypes.data, key.ctypes.data, len(ctr), out.ctypes.data),
           "sdd_debug_philox")
    return out


def sdd_debug_unit_math(w: np.ndarray) -> np.ndarray:
    """(u, ln u, sqrt(-2 ln u), sin 2 pi u, cos 2 pi u) of the path kernel's FP32 Box-Muller
    pieces for each Philox word (n x 5 float32)."""
    w = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1)
    out = np.zeros((len(w), 5), dtype=np.float32)
    _check(lib.sdd_debug_unit_math(w.ctypes.data, len(w), out.ctypes.data), "sdd_debug_unit_math")
    return out


class SddProblem:
    """Owning handle of one problem (context manager); methods forward to the C ABI."""

    def __init__(self, params: SddParams, x0, y0, stream=None):
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.h = sdd_create_problem(params, np.ascontiguousarray(x0, dtype=np.float64)
                                    if isinstance(x0, np.ndarray) else x0,
                                    np.ascontiguousarray(y0, dtype=np.float64)
                                    if isinstance(y0, np.ndarray) else y0, stream)
        self.M = len(sdd_get_interface_nodes(self.h))

    @classmethod
    def load(cls, path: str, stream=None) -> "SddProblem":
        """Resume from a checkpoint written by save() (sdd_load)."""
        self = cls.__new__(cls)
        self.h = 0
        h = sdd_load(path, stream)
        with open(path, "rb") as f:
            head = f.read(12 + ctypes.sizeof(SddParams))
        self.params = SddParams.from_buffer_copy(head[12:])
        self.nx, self.ny = self.params.nx, self.params.ny
        self.h = h
        self.M = len(sdd_get_interface_nodes(self.h))
        return self

    def save(self, path: str) -> None:
        sdd_save(self.h, path)

    def close(self):
        if self.h:
            sdd_destroy_problem(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_monitor(self, omega):
        sdd_set_monitor(self.h, np.ascontiguousarray(omega, dtype=np.float64)
                        if isinstance(omega, np.ndarray) else omega)

    def set_monitor_analytic(self, kind, params):
        sdd_set_monitor_analytic(self.h, kind, params)

    def interface_mc(self):
        est = np.zeros((self.M, 2))
        se = np.zeros((self.M, 2))
        n = np.zeros(self.M, dtype=np.int64)
        status = sdd_interface_mc(self.h, est, se, n)
        return est, se, n, status

    def interface_mc_range(self, node_begin: int, node_end: int, est=None, se=None, n=None):
        """Interface Monte Carlo of nodes node_begin .. node_end - 1 into full-size arrays (created
        when not given); only the range's rows are written."""
        est = np.zeros((self.M, 2)) if est is None else est
        se = np.zeros((self.M, 2)) if se is None else se
        n = np.zeros(self.M, dtype=np.int64) if n is None else n
        status = sdd_interface_mc_range(self.h, node_begin, node_end, est, se, n)
        return est, se, n, status

    def step_from_interface(self, iface):
        x = np.zeros((self.ny, self.nx))
        y = np.zeros((self.ny, self.nx))
        iface = np.ascontiguousarray(iface, dtype=np.float64)
        status = sdd_step_from_interface(self.h, iface, x, y)
        return x, y, status

    def subdomain_solve(self, iface=None):
        x = np.zeros((self.ny, self.nx))
        y = np.zeros((self.ny, self.nx))
        iface = None if iface is None else np.ascontiguousarray(iface, dtype=np.float64)
        status = sdd_subdomain_solve(self.h, iface, x, y)
        return x, y, status

    def step(self):
        x = np.zeros((self.ny, self.nx))
        y = np.zeros((self.ny, self.nx))
        status = sdd_step(self.h, x, y)
        return x, y, status

    def step_mkp(self, K: int):
        x = np.zeros((self.ny, self.nx))
        y = np.zeros((self.ny, self.nx))
        status = sdd_step_mkp(self.h, K, x, y)
        return x, y, status

    def mesh(self):
        x = np.zeros((self.ny, self.nx))
        y = np.zeros((self.ny, self.nx))
        sdd_get_mesh(self.h, x, y)
        return x, y

    def quality(self):
        """Per-cell geometric quality Q (Eq. 8), its maximum and mean, on the current mesh."""
        q = np.zeros((self.ny - 1, self.nx - 1))
        qmax, qmean = ctypes.c_double(), ctypes.c_double()
        _check(lib.sdd_mesh_quality(self.h, q.ctypes.data, ctypes.byref(qmax), ctypes.byref(qmean)),
               "sdd_mesh_quality")
        return q, qmax.value, qmean.value

    def monitor(self):
        w, a, b = (np.zeros((self.ny, self.nx)) for _ in range(3))
        sdd_get_monitor(self.h, w, a, b)
        return w, a, b

    def stats(self):
        return sdd_get_stats(self.h)

    def nodes(self):
        return sdd_get_interface_nodes(self.h)

    def debug_paths(self, node, p_begin, n_paths):
        return sdd_debug_paths(self.h, node, p_begin, n_paths)

    def mc_config(self):
        return sdd_get_mc_config(self.h)

    def set_mc_config(self, threads_per_block=0, blocks_per_sm=0, paths_per_task=0):
        sdd_set_mc_config(self.h, threads_per_block, blocks_per_sm, paths_per_task)

    def tune_mc(self, tune_paths_per_task=True):
        """Time the next step's first path-kernel round over the launch configurations and keep the
        fastest (sdd_tune); returns the chosen configuration."""
        return sdd_tune(self.h, tune_paths_per_task)


def _mc_config(threads_per_block=0, blocks_per_sm=0, paths_per_task=0) -> SddMcConfig:
    c = SddMcConfig()
    c.threads_per_block, c.blocks_per_sm, c.paths_per_task = threads_per_block, blocks_per_sm, paths_per_task
    return c


def sdd_get_mc_config(h: int) -> dict:
    c = SddMcConfig()
    _check(lib.sdd_get_mc_config(h, ctypes.byref(c)), "sdd_get_mc_config")
    return c.as_dict()


def sdd_set_mc_config(h: int, threads_per_block=0, blocks_per_sm=0, paths_per_task=0) -> None:
    c = _mc_config(threads_per_block, blocks_per_sm, paths_per_task)
    _check(lib.sdd_set_mc_config(h, ctypes.byref(c)), "sdd_set_mc_config")


def sdd_tune(h: int, tune_paths_per_task: bool = True) -> dict:
    c = SddMcConfig()
    _check(lib.sdd_tune(h, 1 if tune_paths_per_task else 0, ctypes.byref(c)), "sdd_tune")
    return c.as_dict()


def sdd_batch_get_mc_config(b: int) -> dict:
    c = SddMcConfig()
    _check(lib.sdd_batch_get_mc_config(b, ctypes.byref(c)), "sdd_batch_get_mc_config")
    return c.as_dict()


def sdd_batch_set_mc_config(b: int, threads_per_block=0, blocks_per_sm=0, paths_per_task=0) -> None:
    c = _mc_config(threads_per_block, blocks_per_sm, paths_per_task)
    _check(lib.sdd_batch_set_mc_config(b, ctypes.byref(c)), "sdd_batch_set_mc_config")


def sdd_batch_tune_mc(b: int, tune_paths_per_task: bool = True) -> dict:
    c = SddMcConfig()
    _check(lib.sdd_batch_tune_mc(b, 1 if tune_paths_per_task else 0, ctypes.byref(c)), "sdd_batch_tune_mc")
    return c.as_dict()


def sdd_batch_create(problems, stream=None, use_graph=False) -> int:
    handles = [p.h if isinstance(p, SddProblem) else p for p in problems]
    arr = (ctypes.c_void_p * len(handles))(*handles)
    h = ctypes.c_void_p()
    _check(lib.sdd_batch_create(arr, len(handles), _stream_handle(stream), 1 if use_graph else 0,
                                ctypes.byref(h)), "sdd_batch_create")
    return h.value


def sdd_batch_tune(h: int, threads_per_block: int = 0) -> int:
    chosen = ctypes.c_int32()
    _check(lib.sdd_batch_tune(h, threads_per_block, ctypes.byref(chosen)), "sdd_batch_tune")
    return int(chosen.value)


def sdd_batch_step(b: int) -> None:
    _check(lib.sdd_batch_step(b), "sdd_batch_step")


def sdd_batch_get_stats(b: int) -> dict:
    s = SddStats()
    _check(lib.sdd_batch_get_stats(b, ctypes.byref(s)), "sdd_batch_get_stats")
    return s.as_dict()


def sdd_batch_destroy(b: int) -> None:
    lib.sdd_batch_destroy(b)


class SddBatch:
    """Owning handle of a batch (its problems stay owned by the caller)."""

    def __init__(self, problems, stream=None, use_graph=False):
        self.problems = list(problems)
        self.h = sdd_batch_create(self.problems, stream, use_graph)

    def step(self):
        sdd_batch_step(self.h)

    def tune(self, threads_per_block: int = 0) -> int:
        """Path-kernel block size: 128, 256 or 512, or 0 to time all three and keep the fastest."""
        return sdd_batch_tune(self.h, threads_per_block)

    def stats(self):
        return sdd_batch_get_stats(self.h)

    def mc_config(self):
        return sdd_batch_get_mc_config(self.h)

    def set_mc_config(self, threads_per_block=0, blocks_per_sm=0, paths_per_task=0):
        sdd_batch_set_mc_config(self.h, threads_per_block, blocks_per_sm, paths_per_task)

    def tune_mc(self, tune_paths_per_task=True):
        return sdd_batch_tune_mc(self.h, tune_paths_per_task)

    def close(self):
        if self.h:
            sdd_batch_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------------------
# Serving (continuous batching of one-step requests).
# --------------------------------------------------------------------------------------

def sdd_server_create(params: SddServerParams, stream) -> int:
    h = ctypes.c_void_p()
    _check(lib.sdd_server_create(ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)),
           "sdd_server_create")
    return h.value


def sdd_server_submit(s: int, params: SddParams, x0, y0, monitor_kind: int = SDD_MONITOR_NODAL,
                      monitor_params=None, omega=None, step_index: int = 0) -> int:
    mp = None if monitor_params is None else np.ascontiguousarray(monitor_params, dtype=np.float64)
    n = 0 if mp is None else int(mp.size)
    rid = ctypes.c_int64()
    _check(lib.sdd_server_submit(s, ctypes.byref(params), _ptr(x0), _ptr(y0), monitor_kind, _ptr(mp), n,
                                 _ptr(omega), step_index, ctypes.byref(rid)), "sdd_server_submit")
    return rid.value


def sdd_server_progress(s: int):
    nr, nq = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.sdd_server_progress(s, ctypes.byref(nr), ctypes.byref(nq)), "sdd_server_progress")
    return nr.value, nq.value


def sdd_server_poll(s: int, cap: int = 1024):
    ids = np.zeros(max(cap, 1), dtype=np.int64)
    n = ctypes.c_int32()
    _check(lib.sdd_server_poll(s, _ptr(ids), cap, ctypes.byref(n)), "sdd_server_poll")
    return [int(v) for v in ids[:n.value]]


def sdd_server_result(s: int, rid: int, x=None, y=None, est_xy=None, se_xy=None,
                      ok=(SDD_OK, SDD_ERR_SE_NOT_REACHED)):
    st = SddStats()
    status = _check(lib.sdd_server_result(s, rid, _ptr(x), _ptr(y), _ptr(est_xy), _ptr(se_xy),
                                          ctypes.byref(st)), "sdd_server_result", ok=ok)
    return status, st.as_dict()


def sdd_server_cancel(s: int, rid: int) -> None:
    _check(lib.sdd_server_cancel(s, rid), "sdd_server_cancel")


def sdd_server_get_stats(s: int) -> dict:
    o = SddServerStats()
    _check(lib.sdd_server_get_stats(s, ctypes.byref(o)), "sdd_server_get_stats")
    return o.as_dict()


def sdd_server_destroy(s: int) -> None:
    lib.sdd_server_destroy(s)


class SddServer:
    """Owning handle of a server; results come back as numpy arrays."""

    def __init__(self, params: SddServerParams, stream):
        self.h = sdd_server_create(params, stream)
        self.shapes = {}

    def submit(self, params: SddParams, x0, y0, monitor_kind=SDD_MONITOR_NODAL, monitor_params=None,
               omega=None, step_index=0) -> int:
        rid = sdd_server_submit(self.h, params, x0, y0, monitor_kind, monitor_params, omega, step_index)
        M = int(sdd_interface_layout(params.nx, params.ny, params.px, params.py, params.periodic).shape[0])
        self.shapes[rid] = (params.nx, params.ny, M)
        return rid

    def progress(self):
        return sdd_server_progress(self.h)

    def poll(self, cap=1024):
        return sdd_server_poll(self.h, cap)

    def result(self, rid, ok=(SDD_OK, SDD_ERR_SE_NOT_REACHED)):
        nx, ny, M = self.shapes.pop(rid)
        x = np.empty((ny, nx))
        y = np.empty((ny, nx))
        est = np.empty((max(M, 1), 2))
        se = np.empty((max(M, 1), 2))
        status, st = sdd_server_result(self.h, rid, x, y, est, se, ok=ok)
        return {"x": x, "y": y, "est": est[:M], "se": se[:M], "stats": st, "status": status}

    def cancel(self, rid):
        sdd_server_cancel(self.h, rid)

    def stats(self):
        return sdd_server_get_stats(self.h)

    def close(self):
        if self.h:
            sdd_server_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------------------
# Checkpoint / resume.
# --------------------------------------------------------------------------------------

def sdd_save(h: int, path: str) -> None:
    _check(lib.sdd_save(h, os.fsencode(path)), "sdd_save")


def sdd_load(path: str, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib.sdd_load(os.fsencode(path), _stream_handle(stream), ctypes.byref(h)), "sdd_load")
    return h.value
