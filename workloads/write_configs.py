"""Writes workloads/configs.json: the benchmark configurations as plain data, for users of the C
ABI who do not use Python.  The file mirrors the definitions in workloads/__init__.py exactly;
tests/test_workloads_json.py checks that it is current.

    python workloads/write_configs.py
"""
import dataclasses
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import workloads as W  # noqa: E402


def configs() -> dict:
    d = dataclasses.asdict
    return {
        "C0_dirichlet33_2x2_gauss_fp64": d(W.c0_small_fp64()),
        "C1_front257_4x4": d(W.c1_front(W.PREC_FP32_KAHAN).replace(se_target=1e-4, max_paths_per_node=1 << 25)),
        "C1_front257_4x4_periodic": d(W.c1_front(W.PREC_FP32_KAHAN, periodic=1).replace(
            se_target=1e-4, max_paths_per_node=1 << 25)),
        "C2_sine257_4x4": d(W.c2_sine()),
        "C3_mix64": [d(p.replace(precision=W.PREC_FP32_KAHAN)) for p in W.c3_mix(64, paths=10000)],
        "C4_serving": {
            "requests": "the C3 shapes and bump monitors drawn with seed 777 (c3_mix(n, seed=777)), "
                        "one step each at se_target 1e-4, first chunk 1e4 paths per node",
            "arrivals": {"process": "poisson", "rate_per_s": 2000.0, "seed": 7, "n_requests": 10000},
            "mem_budget_gb": 150.0,
        },
        "five_ring41": {str(k): d(W.five_ring(k)) for k in (2, 3, 4)},
    }


def main() -> None:
    with open(os.path.join(HERE, "configs.json"), "w") as f:
        json.dump(configs(), f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
