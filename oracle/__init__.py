"""CPU oracle of the stochastic domain decomposition (SDD) mesh generator.

TEST INFRASTRUCTURE.  Only tests/, the package's smoke check (__graft_entry__.smoke) and
bench.py's CPU-baseline leg may import, call, link or execute anything here.  The product
path (the CUDA library and its Python binding) never does, and shares no code with it.

Plain, slow, obviously correct restatements of the paper (Bihlo, Haynes & Walsh,
"Stochastic domain decomposition for time dependent adaptive mesh generation"):
  _clib / sdd_oracle.c   Philox4x32-10, Box-Muller, interpolation, one Euler-Maruyama path
                         with the boundary test (Eq. 5a, 5b, 6, 7; Sec. 3.4), estimator sums
  monitor.py             omega on the current mesh and its FD gradient (Sec. 2, 3.2, 3.4)
  layout.py              interface nodes and subdomains (Sec. 3.1, 3.5)
  mc.py                  node estimates, SE, adaptive path counts (Sec. 3.4)
  solve.py               backward-Euler 5-point subdomain / single-domain solves (Sec. 3.5)
  step.py                one alternating step (Sec. 3.6)
Every function is pinned by tests/test_oracle_*.py against closed forms, invariants,
published known-answer vectors, library routines or brute force.
"""
from . import _clib, layout, mc, monitor, solve, step  # noqa: F401

build = _clib.build
