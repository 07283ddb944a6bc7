"""Bounds-checked build (-DSDD_BOUNDS_CHECK): every monitor, mesh, boundary and queue index of the
path kernel is checked before its load, and an index outside its array is counted instead of
read.  Workloads covering Dirichlet and periodic grids, both generator forms, bicubic and bilinear
terminal values, the bridge on and off, a moving boundary, uneven splits, interface sampling, a
3x3 grid, the chaotic 257x257 front over two steps, and a batch run through the checked library
in a child process, and meet no out-of-range index.  The normal library carries no checks."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, "tests")
    import torch
    import paper_1504_00084_gb300 as S
    import workloads as W
    from gpu_helpers import gpu_problem
    from test_gpu_batch import small_mix

    c0 = W.c0_small_fp64()
    cases = [
        c0,
        c0.replace(precision=W.PREC_FP32_KAHAN, paths_per_node=4096),
        c0.replace(nx=17, ny=17, periodic=1, tau=1.0, Lx=2.0, monitor_params=[6.0, 40.0, 0.3, 0.6]),
        c0.replace(form=W.FORM_WINSLOW, tau=1.0, bicubic=0, bb_test=0),
        c0.replace(moving_boundary=1, monitor_params=[10.0, 8.0, 0.5, 0.2]),
        c0.replace(px=3, py=5, iface_stride=3),
        c0.replace(nx=3, ny=3, px=2, py=2, paths_per_node=3000),
        W.c1_front(W.PREC_FP32_KAHAN).replace(paths_per_node=4096),
        W.c1_front(W.PREC_FP32_KAHAN, periodic=1).replace(paths_per_node=2048),
    ]
    for prob in cases:
        h = gpu_problem(prob)
        h.step()
        h.step()
        if h.M > 0:
            h.debug_paths(h.M - 1, 0, 256)
        h.close()
    probs = small_mix(W.PREC_FP32_KAHAN, paths=2048, n=6)
    hs = [gpu_problem(p) for p in probs]
    with S.SddBatch(hs, stream=torch.cuda.Stream()) as b:
        b.step()
        b.step()
        b.stats()
    for h in hs:
        h.close()
    print("violations", S.sdd_debug_bounds_violations())
""")


def test_checked_build_meets_no_out_of_range_index():
    import paper_1504_00084_gb300 as S
    from paper_1504_00084_gb300 import build as B
    assert S.sdd_debug_bounds_violations() == -1   # the normal build has no checks
    lib = B.build(bounds_check=True)
    env = dict(os.environ, SDD_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    last = r.stdout.strip().splitlines()[-1].split()
    assert last[0] == "violations" and int(last[1]) == 0, r.stdout[-2000:]
