"""Builds and loads the oracle's C core (sdd_oracle.c) -- TEST INFRASTRUCTURE.

Compiled with gcc, -ffp-contract=off (no fused multiply-add on any host, x86-64 or Arm),
OpenMP over interface nodes.  The shared object goes to oracle/_build/ (git-ignored).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "sdd_oracle.c"), os.path.join(HERE, "oracle_paths_body.h")]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C core if it is missing or older than its sources."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, os.path.join(HERE, "sdd_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _problem_struct(real):
    fields = [(n, ctypes.c_int32) for n in ("nx", "ny", "periodic", "form", "K", "bicubic",
                                            "bb_test", "tstep")]
    fields += [("key0", ctypes.c_uint32), ("key1", ctypes.c_uint32)]
    fields += [(n, ctypes.c_double) for n in ("Lx", "Ly", "tau", "dt")]
    fields += [(n, ctypes.POINTER(real)) for n in ("w", "w_xi", "w_eta", "X", "Y", "bnd")]

    class OracleProblem(ctypes.Structure):
        _fields_ = fields

    return OracleProblem


ProblemF64 = _problem_struct(ctypes.c_double)
ProblemF32 = _problem_struct(ctypes.c_float)

P = ctypes.c_void_p
I32, I64, U32, F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            L.oracle_philox4x32_10.argtypes = [P, P, P]
            L.oracle_philox_batch.argtypes = [I64, P, P, P]
            L.oracle_max_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            for sfx, st in (("f64", ProblemF64), ("f32", ProblemF32)):
                getattr(L, f"oracle_path_{sfx}").argtypes = [ctypes.POINTER(st), U32, ctypes.c_int,
                                                             ctypes.c_int, U32, P, P, P, P, P]
                getattr(L, f"oracle_paths_{sfx}").argtypes = [ctypes.POINTER(st), U32, ctypes.c_int,
                                                              ctypes.c_int, I64, I64, P, P, P, P]
                getattr(L, f"oracle_interface_sums_{sfx}").argtypes = [ctypes.POINTER(st), I64, P, P,
                                                                       P, P, P, P, P]
                getattr(L, f"oracle_box_muller_{sfx}").argtypes = [U32, U32, P, P]
                getattr(L, f"oracle_uniform_{sfx}").argtypes = [U32]
                getattr(L, f"oracle_uniform_{sfx}").restype = F64
                getattr(L, f"oracle_interp_{sfx}").argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                               ctypes.c_int, P, I64, P, P]
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)
