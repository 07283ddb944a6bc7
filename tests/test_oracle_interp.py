"""Pins of the oracle's interpolation (Sec. 3.4: bilinear for the monitor, bicubic for the mesh)."""
import numpy as np
import pytest

from oracle import _clib


def interp(f, pts, periodic=0, bicubic=0, real=np.float64):
    L = _clib.lib()
    f = np.ascontiguousarray(f, dtype=real)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    out = np.zeros(len(pts))
    sfx = "f32" if real is np.float32 else "f64"
    ny, nx = f.shape
    getattr(L, f"oracle_interp_{sfx}")(nx, ny, periodic, bicubic, _clib.ptr(f), len(pts),
                                       _clib.ptr(pts), _clib.ptr(out))
    return out


def grid(nx, ny):
    xi = np.arange(nx) / (nx - 1)
    eta = np.arange(ny) / (ny - 1)
    return np.meshgrid(xi, eta)


@pytest.mark.parametrize("nx,ny", [(3, 3), (9, 5), (33, 17)])
def test_bilinear_reproduces_bilinear_functions(oracle_lib, nx, ny):
    XI, ETA = grid(nx, ny)
    f = lambda a, b: 0.3 + 1.7 * a - 2.1 * b + 0.9 * a * b
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, size=(500, 2))
    pts[:4] = [[0, 0], [1, 1], [0, 1], [1, 0]]
    got = interp(f(XI, ETA), pts)
    assert np.allclose(got, f(pts[:, 0], pts[:, 1]), atol=1e-13)


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 7), (33, 17)])
def test_keys_bicubic_reproduces_quadratics_with_boundary_rule(oracle_lib, nx, ny):
    """Keys' a = -1/2 kernel with his boundary extrapolation is exact for quadratics (Keys 1981)."""
    XI, ETA = grid(nx, ny)
    f = lambda a, b: 1 + 2 * a - 3 * b + 0.5 * a * a + 0.7 * a * b - 1.3 * b * b
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 1, size=(500, 2))
    pts[:6] = [[0, 0], [1, 1], [0, 1], [1, 0], [1e-9, 0.5], [0.5, 1 - 1e-9]]
    got = interp(f(XI, ETA), pts, bicubic=1)
    assert np.allclose(got, f(pts[:, 0], pts[:, 1]), atol=1e-12)


def test_keys_bicubic_not_exact_for_cubics_but_third_order(oracle_lib):
    """Cubic convolution with a = -1/2 converges at O(h^3) on a smooth periodic field."""
    errs = []
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, size=(400, 2))
    g = lambda a, b: np.sin(2 * np.pi * a) * np.cos(2 * np.pi * b) + 0.3 * np.sin(4 * np.pi * b)
    for n in (17, 33, 65):
        XI, ETA = grid(n, n)
        errs.append(np.abs(interp(g(XI, ETA), pts, periodic=1, bicubic=1) - g(pts[:, 0], pts[:, 1])).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.0 < r1 < 20.0 and 6.0 < r2 < 20.0, errs


def test_periodic_interp_wraps(oracle_lib):
    n = 17
    XI, ETA = grid(n, n)
    rng = np.random.default_rng(4)
    f = rng.normal(size=(n, n))
    f[:, -1] = f[:, 0]
    f[-1, :] = f[0, :]
    pts = rng.uniform(0, 1, size=(200, 2))
    for bic in (0, 1):
        a = interp(f, pts, periodic=1, bicubic=bic)
        for shift in ([1, 0], [0, -1], [3, 2], [-2, -5]):
            b = interp(f, pts + np.array(shift, float), periodic=1, bicubic=bic)
            assert np.allclose(a, b, atol=1e-12)
    # at the nodes both interpolants return the nodal values
    nodes = np.stack([XI.ravel(), ETA.ravel()], 1)
    for bic in (0, 1):
        assert np.allclose(interp(f, nodes, periodic=1, bicubic=bic), f.ravel(), atol=1e-12)
        assert np.allclose(interp(f, nodes, periodic=0, bicubic=bic), f.ravel(), atol=1e-12)


def test_float_variant_close_to_double(oracle_lib):
    n = 33
    XI, ETA = grid(n, n)
    f = np.exp(XI) * np.cos(ETA)
    pts = np.random.default_rng(5).uniform(0, 1, size=(300, 2))
    for bic in (0, 1):
        a = interp(f, pts, bicubic=bic)
        b = interp(f, pts, bicubic=bic, real=np.float32)
        assert np.abs(a - b).max() < 64 * np.finfo(np.float32).eps * np.abs(a).max()
