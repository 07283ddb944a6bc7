"""The library's host code (argument validation, interface layout and sampling tables, adaptive
schedule, checkpoint parsing, status strings) under AddressSanitizer and UBSan: the host-side
ABI tests run in a child process against a build whose host code carries both sanitizers, with
libasan preloaded, and finish with no report.  Needs no GPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    try:
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True,
                              timeout=60).stdout.strip()
    except (OSError, subprocess.SubprocessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_host_abi_under_address_and_undefined_behaviour_sanitizers():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc's sanitizer runtimes are not installed")
    sys.path.insert(0, ROOT)
    from paper_1504_00084_gb300 import build as B
    lib = B.build(sanitize=True)
    env = dict(os.environ, SDD_LIB_PATH=lib, LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0,protect_shadow_gap=0,abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1,halt_on_error=1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join("tests", "test_abi_host.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "ERROR: AddressSanitizer" not in out and "runtime error:" not in out, out[-4000:]
