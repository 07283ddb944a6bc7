"""Seeded synthetic inputs for the stochastic domain decomposition (SDD) mesh generator.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's tests.
It holds only problem descriptions and seeded random draws of their parameters
(grid sizes, subdomain splits, monitor parameters, initial meshes, arrival times).
It contains none of the method's arithmetic: no monitor evaluation, no paths, no
solves.  Every workload is a synthetic stand-in shaped like the paper's own
experiments (Sec. 4: 41x41 grids, analytic mesh densities, N = 1e3..1e4 paths),
scaled to the sizes listed below.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# Monitor kinds (the mesh density omega evaluated on the current physical mesh).
MONITOR_NODAL = 0   # nodal values supplied by the caller
MONITOR_GAUSS = 1   # sqrt(1 + a exp(-b |x - c|^2))                    params (a, b, cx, cy)
MONITOR_FRONT = 2   # sqrt(1 + alpha |grad u|^2), u = tanh(R (r - r0 - v t))  params (alpha, R, r0, v, cx, cy)
MONITOR_BUMPS = 3   # 1 + sum_i a_i exp(-|x - c_i|^2 / w_i^2)          params (a_1, w_1, cx_1, cy_1, a_2, ...)
MONITOR_RINGS = 4   # sqrt(1 + alpha |grad u|^2), u = sum_k tanh(R (|x - c_k|^2 - r2))  params (alpha, R, r2, cx_1, cy_1, ...)

FORM_DIV = 0        # tau x_t = div(omega grad x)
FORM_WINSLOW = 1    # tau x_t = (grad omega / omega) . grad x + lap x   (the paper's Eq. for the generator)

PREC_FP64 = 0       # paths and accumulation in FP64
PREC_FP32_ACC64 = 1 # paths in FP32, estimator sums in FP64
PREC_FP32_KAHAN = 2 # paths in FP32, Kahan-compensated FP32 estimator sums


@dataclass
class Problem:
    """One mesh problem: grid, split, generator parameters and the monitor."""
    name: str
    nx: int
    ny: int
    px: int
    py: int
    periodic: int = 0
    form: int = FORM_DIV
    precision: int = PREC_FP64
    bicubic: int = 1
    bb_test: int = 1
    Lx: float = 1.0
    Ly: float = 1.0
    tau: float = 1e-2
    dt: float = 1e-2
    substeps: int = 100
    seed: int = 1
    paths_per_node: int = 1000
    se_target: float = 0.0
    max_paths_per_node: int = 0
    solve_rtol: float = 1e-12
    solve_max_iter: int = 20000
    iface_stride: int = 0          # > 1: Monte Carlo at every k-th node of each interface line
    subdomain_scheme: int = 0      # 0 backward Euler, 1 forward Euler (the paper's, Sec. 3.5)
    fe_max_substeps: int = 0       # forward Euler: refuse more substeps than this (0: 2^16)
    moving_boundary: int = 0       # 1: tangential boundary coordinates follow the 1-D generator
    monitor_kind: int = MONITOR_GAUSS
    monitor_params: List[float] = field(default_factory=list)
    steps: int = 1
    t0: float = 0.0

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def identity_mesh(p: Problem):
    """Uniform initial mesh x = Lx xi, y = Ly eta on the (ny, nx) node grid (row-major, eta slow)."""
    xi = np.arange(p.nx, dtype=np.float64) / (p.nx - 1)
    eta = np.arange(p.ny, dtype=np.float64) / (p.ny - 1)
    x = np.broadcast_to(p.Lx * xi[None, :], (p.ny, p.nx)).copy()
    y = np.broadcast_to(p.Ly * eta[:, None], (p.ny, p.nx)).copy()
    return x, y


def sine_mode_mesh(p: Problem, amp: float = 0.05, periodic_mode: bool = False):
    """Identity mesh plus one Fourier mode of the displacement (closed-form decay tests).

    Dirichlet: amp sin(pi xi) sin(pi eta) on both components (vanishes on the boundary).
    Periodic:  amp sin(2 pi xi) sin(2 pi eta) (periodic displacement).
    """
    x, y = identity_mesh(p)
    xi = np.arange(p.nx, dtype=np.float64) / (p.nx - 1)
    eta = np.arange(p.ny, dtype=np.float64) / (p.ny - 1)
    k = 2.0 if periodic_mode else 1.0
    mode = amp * np.outer(np.sin(k * np.pi * eta), np.sin(k * np.pi * xi))
    return x + mode, y + mode


# --------------------------------------------------------------------------------------
# Named workloads (sizes from the project's benchmark plan).
# --------------------------------------------------------------------------------------

def c0_small_fp64() -> Problem:
    """33x33 grid, 2x2 subdomains (61 interface nodes), tau = dt = 1e-2, 1000 paths,
    ds = 1e-4 (K = 100), Gaussian monitor sqrt(1 + 10 exp(-50 |x - (1/2,1/2)|^2)), FP64, one step."""
    return Problem(name="dirichlet33_2x2_gauss_fp64", nx=33, ny=33, px=2, py=2,
                   tau=1e-2, dt=1e-2, substeps=100, seed=1, paths_per_node=1000,
                   precision=PREC_FP64, monitor_kind=MONITOR_GAUSS,
                   monitor_params=[10.0, 50.0, 0.5, 0.5], steps=1)


def c1_front(precision: int = PREC_FP32_ACC64, periodic: int = 0) -> Problem:
    """257x257 grid, 4x4 subdomains (1521 interface nodes; 2032 periodic), 1e5 paths per node,
    ds = 1e-5 (K = 100), dt = 1e-3, tau = 1e-2, moving-front monitor
    u = tanh(50 (r - 0.25 - 0.1 t)), omega = sqrt(1 + 50 |grad u|^2), 20 time steps."""
    return Problem(name="front257_4x4" + ("_periodic" if periodic else ""), nx=257, ny=257,
                   px=4, py=4, periodic=periodic, tau=1e-2, dt=1e-3, substeps=100, seed=1,
                   paths_per_node=100000, precision=precision, monitor_kind=MONITOR_FRONT,
                   monitor_params=[50.0, 50.0, 0.25, 0.1, 0.5, 0.5], steps=20,
                   solve_rtol=1e-10)


def c2_sine(precision: int = PREC_FP32_ACC64, paths: int = 1000) -> Problem:
    """Precision sweep case: 257x257 / 4x4, omega = 1, initial mesh xi + 0.05 sin(pi xi) sin(pi eta);
    closed form xi + 0.05 exp(-2 pi^2 t / tau) sin(pi xi) sin(pi eta)."""
    return Problem(name="sine257_4x4", nx=257, ny=257, px=4, py=4, tau=1e-2, dt=1e-3,
                   substeps=100, seed=1, paths_per_node=paths, precision=precision,
                   monitor_kind=MONITOR_BUMPS, monitor_params=[], steps=1, solve_rtol=1e-10)


def five_ring(px: int, steps: int = 100, paths: int = 10000, nx: int = 41) -> Problem:
    """The periodic five-ring problem of the paper's Sec. 4.2: u = sum of five tanh(R (|x - c|^2 - 1/8))
    rings, R = 30, on [-1, 1)^2 (here shifted to [0, 2)^2, centres (1,1), (1/2,1/2), (1/2,3/2),
    (3/2,1/2), (3/2,3/2)), arc-length monitor sqrt(1 + 0.2 |grad u|^2), 41 x 41 nodes,
    dt = 5e-4 up to t = 0.05 (100 steps), one Euler-Maruyama substep per step, 1e4 paths, the
    paper's generator form (tau = 1)."""
    centres = [1.0, 1.0, 0.5, 0.5, 0.5, 1.5, 1.5, 0.5, 1.5, 1.5]
    return Problem(name=f"five_ring{nx}_{px}x{px}", nx=nx, ny=nx, px=px, py=px, periodic=1,
                   form=FORM_WINSLOW, precision=PREC_FP64, Lx=2.0, Ly=2.0, tau=1.0, dt=5e-4,
                   substeps=1, seed=1, paths_per_node=paths, monitor_kind=MONITOR_RINGS,
                   monitor_params=[0.2, 30.0, 0.125] + centres, steps=steps, solve_rtol=1e-12)


GRID_CHOICES = (65, 129, 257, 513)
SPLIT_CHOICES = (2, 4, 8)


def c3_mix(n_problems: int = 64, seed: int = 12345, paths: int = 10000) -> List[Problem]:
    """Batched mix of independent problems: grids from {65,129,257,513}^2, splits from
    {2x2,4x4,8x8}, monitor = 1 + sum of 1..4 Gaussian bumps with amplitude U[1,20],
    width U[0.02,0.1], centre U[0.1,0.9]^2; tau = 1e-2, dt = 1e-3, ds = 1e-5, FP32 paths.
    Path seed of problem k is k + 1."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        n = int(rng.choice(GRID_CHOICES))
        s = int(rng.choice(SPLIT_CHOICES))
        nb = int(rng.integers(1, 5))
        params: List[float] = []
        for _ in range(nb):
            a = float(rng.uniform(1.0, 20.0))
            w = float(rng.uniform(0.02, 0.1))
            cx, cy = (float(v) for v in rng.uniform(0.1, 0.9, size=2))
            params += [a, w, cx, cy]
        out.append(Problem(name=f"mix{k:02d}_{n}_{s}x{s}", nx=n, ny=n, px=s, py=s, tau=1e-2,
                           dt=1e-3, substeps=100, seed=k + 1, paths_per_node=paths,
                           precision=PREC_FP32_ACC64, monitor_kind=MONITOR_BUMPS,
                           monitor_params=params, steps=1, solve_rtol=1e-10))
    return out


def poisson_arrivals(n_requests: int = 10000, rate_per_s: float = 2000.0, seed: int = 7):
    """Arrival times (seconds) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))
