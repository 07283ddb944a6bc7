"""bench.py's JSON line contract, checked on the CPU through the reference arm (the oracle timed
on the host cores): one line with the metric, value, unit, counts, config, the cpu_baseline
object and an e2e object; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-seconds", "2"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return [line for line in r.stdout.splitlines() if line.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    d = json.loads(lines[-1])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "config", "dtype", "scaling"):
        assert isinstance(d[key], (str, dict)) and d[key]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["single_core"]["path_steps_per_s"] > 0 and 0 < cb["sigma_v"]["mean"] <= cb["sigma_v"]["max"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_clock_sampler_reports_the_timed_window_only():
    """The clock record reports the samples time-stamped inside the timed window (nvidia-smi's
    timestamp column), here a clock stuck low before the window and a throttle reason after it."""
    import datetime
    import tempfile
    import time

    sys.path.insert(0, ROOT)
    import bench

    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    t0 = time.time()
    for k in range(12):
        ts = datetime.datetime.fromtimestamp(t0 + 0.2 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        mhz = 1000 if k < 3 else 2070
        thermal = "Active" if k >= 10 else "Not Active"
        cs.f.write(f"{ts}, 0, {mhz}, 2070, 500.0, 0x0, Not Active, {thermal}, Not Active, Not Active\n")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    cs.p = _Done()
    c = cs.stop((t0 + 0.5, t0 + 1.9))
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 7}


def test_roofline_basis_follows_the_problem_switches():
    """The algorithmic count drops the exit tests a path does not take (Sec. 3.4: a periodic path
    has no boundary, and the bridge test is a switch), and the ncu-derived instruction and DRAM
    figures are reported only for the kernel they were taken on."""
    import argparse

    sys.path.insert(0, ROOT)
    import bench
    import workloads as W

    front = W.c1_front(W.PREC_FP32_KAHAN)
    assert bench.ops_per_path_step(front) == bench.OPS_PER_PATH_STEP == 158
    assert bench.ops_per_path_step(front.replace(bb_test=0)) == 158 - 28 - 3
    assert bench.ops_per_path_step(front.replace(periodic=1)) == 158 - 6 - 28 - 3
    args = argparse.Namespace(precision="kahan", iface_stride=0)
    assert bench.counters_apply(front, args)
    for other in (front.replace(periodic=1), front.replace(bb_test=0), front.replace(form=1),
                  front.replace(bicubic=0)):
        assert not bench.counters_apply(other, args)
    assert not bench.counters_apply(front, argparse.Namespace(precision="fp64", iface_stride=0))
    assert not bench.counters_apply(front, argparse.Namespace(precision="kahan", iface_stride=4))
