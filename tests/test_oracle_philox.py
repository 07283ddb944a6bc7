"""Pins of the oracle's random numbers: Philox4x32-10 and the uniform/normal transforms."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.stats

from oracle import _clib

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def philox(ctr, key):
    L = _clib.lib()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    L.oracle_philox_batch(len(ctr), _clib.ptr(ctr), _clib.ptr(key), _clib.ptr(out))
    return out


def test_philox_known_answer_vectors(oracle_lib):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox(v[0:4], v[4:6])[0]
        assert list(out) == v[6:10]


_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
from triton.language.random import philox_impl
@triton.jit
def k(c_ptr, k_ptr, o_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4*i); c1 = tl.load(c_ptr + 4*i+1); c2 = tl.load(c_ptr + 4*i+2); c3 = tl.load(c_ptr + 4*i+3)
    k0 = tl.load(k_ptr + 2*i); k1 = tl.load(k_ptr + 2*i+1)
    a, b, c, d = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(o_ptr + 4*i, a); tl.store(o_ptr + 4*i+1, b); tl.store(o_ptr + 4*i+2, c); tl.store(o_ptr + 4*i+3, d)
d = json.load(sys.stdin)
c = torch.tensor(np.array(d["ctr"], dtype=np.uint32).view(np.int32)).view(torch.uint32)
kk = torch.tensor(np.array(d["key"], dtype=np.uint32).view(np.int32)).view(torch.uint32)
o = torch.zeros_like(c)
k[(1,)](c, kk, o, N=c.shape[0])
print(json.dumps(o.view(torch.int32).numpy().view(np.uint32).tolist()))
"""


def test_philox_matches_library_implementation(oracle_lib):
    """Cross-check against Triton's Philox4x32-10 (a library routine), run by its CPU interpreter."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(64, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = [5, 7, 11, 0]
    key[0] = [1, 0]
    env = dict(os.environ, TRITON_INTERPRET="1")
    try:
        res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(
            {"ctr": ctr.tolist(), "key": key.tolist()}), capture_output=True, text=True,
            timeout=600, env=env)
    except subprocess.TimeoutExpired:
        pytest.skip("triton interpreter timed out")
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr.strip().splitlines()[-1][:200])
    ref = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint32)
    assert np.array_equal(philox(ctr, key), ref)


def test_uniforms_are_exact_and_open(oracle_lib):
    L = oracle_lib
    # FP64: (w + 1/2) 2^-32, FP32: (floor(w/2^9) + 1/2) 2^-23 -- closed forms at the ends.
    assert L.oracle_uniform_f64(0) == 2.0 ** -33
    assert L.oracle_uniform_f64(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    assert L.oracle_uniform_f32(0) == 2.0 ** -24
    assert L.oracle_uniform_f32(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert L.oracle_uniform_f32(511) == 2.0 ** -24       # same 23-bit bucket as 0
    assert L.oracle_uniform_f32(512) == 3 * 2.0 ** -24


@pytest.mark.parametrize("sfx", ["f64", "f32"])
def test_box_muller_normal(oracle_lib, sfx):
    """Box-Muller output is N(0,1): moments, Kolmogorov-Smirnov, independence, polar identity."""
    L = oracle_lib
    n = 100000
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(n)
    w = philox(ctr, np.tile(np.array([7, 0], np.uint32), (n, 1)))
    fn = getattr(L, f"oracle_box_muller_{sfx}")
    z = np.zeros((n, 2))
    a, b = ctypes.c_double(), ctypes.c_double()
    for q in range(n):
        fn(int(w[q, 0]), int(w[q, 1]), ctypes.byref(a), ctypes.byref(b))
        z[q] = a.value, b.value
    for c in range(2):
        assert abs(z[:, c].mean()) < 5 / np.sqrt(n)
        assert abs(z[:, c].var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert scipy.stats.kstest(z[:, c], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5 / np.sqrt(n)
    # polar identity: z1^2 + z2^2 = -2 ln u1, angle = 2 pi u2
    u1 = np.array([getattr(L, f"oracle_uniform_{sfx}")(int(v)) for v in w[:200, 0]])
    u2 = np.array([getattr(L, f"oracle_uniform_{sfx}")(int(v)) for v in w[:200, 1]])
    tol = 1e-12 if sfx == "f64" else 2e-5
    assert np.allclose(z[:200, 0] ** 2 + z[:200, 1] ** 2, -2 * np.log(u1), rtol=tol, atol=tol)
    ang = np.mod(np.arctan2(z[:200, 1], z[:200, 0]), 2 * np.pi)
    d = np.abs(ang - 2 * np.pi * u2)
    d = np.minimum(d, 2 * np.pi - d)
    assert d.max() < (1e-9 if sfx == "f64" else 1e-4)
