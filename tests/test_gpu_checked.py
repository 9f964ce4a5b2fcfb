"""The bounds-checked build (HEAT1D_CHECKED) on the GPU.

Every checked index test in the kernels records HEAT1D_ERR_BOUNDS in the
run's status word and skips the access instead of trapping.  The checked
library's self-test shows that a checked load and store one past the end of a
buffer are caught; then the small-case GPU suites of the on-chip synchronous,
per-step asynchronous (with and without clusters), blocked, periodic,
resumed, streamed asynchronous and batched runs are run again against the
checked library (a child pytest with HEAT1D_CHECKED=1), where they must pass
bit for bit with no status raised.
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def child(args, timeout):
    env = dict(os.environ, HEAT1D_CHECKED="1")
    return subprocess.run([sys.executable] + args, cwd=ROOT, env=env, timeout=timeout, capture_output=True, text=True)


def test_checked_library_catches_an_out_of_bounds_index():
    code = ("from paper_1510_08982_gb300 import build, heat1d; build.build(); "
            "print(int(heat1d.checked()), heat1d.checked_selftest())")
    p = child(["-c", code], 900)
    assert p.returncode == 0, p.stdout + p.stderr
    checked, st = p.stdout.split()[-2:]
    assert checked == "1"
    assert int(st) == -7  # HEAT1D_ERR_BOUNDS


def test_small_gpu_suites_pass_under_the_checked_build():
    suites = ["tests/test_gpu_parity.py", "tests/test_gpu_cluster.py", "tests/test_gpu_blocked.py",
              "tests/test_gpu_periodic.py", "tests/test_gpu_resume.py", "tests/test_gpu_batched.py",
              "tests/test_gpu_stream_async.py"]
    skip = "not full_size and not full_horizon and not default_tiles and not uneven_rods_workload"
    p = child(["-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu", "-k", skip] + suites, 1800)
    print(p.stdout[-3000:])
    assert p.returncode == 0, p.stdout[-6000:] + p.stderr[-3000:]
