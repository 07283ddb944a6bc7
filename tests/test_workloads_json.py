"""workloads/configs.json (the benchmark configurations as plain data) is current: it equals the
Python definitions it mirrors, and every problem in it rebuilds a workloads.Problem."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_configs_json_is_current_and_rebuilds_problems():
    sys.path.insert(0, os.path.join(ROOT, "workloads"))
    import write_configs
    import workloads as W
    with open(os.path.join(ROOT, "workloads", "configs.json")) as f:
        stored = json.load(f)
    assert stored == json.loads(json.dumps(write_configs.configs()))
    assert W.Problem(**stored["C1_front257_4x4"]) == W.c1_front(W.PREC_FP32_KAHAN).replace(
        se_target=1e-4, max_paths_per_node=1 << 25)
    mix = [W.Problem(**p) for p in stored["C3_mix64"]]
    assert len(mix) == 64 and {p.nx for p in mix} <= {65, 129, 257, 513}
