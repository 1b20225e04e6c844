"""Runs GPU parity, time-parallel and serving cases against the library built
with -DDSP_BOUNDS_CHECK: every device index that the normal build leaves
unchecked (table ranges staged by a launch, a CTA's tile) is verified, and an
out-of-range one would surface as DSP_E_BOUNDS and fail those tests.  The
library checks its own indexes here, in place of an external memory checker."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_suite_under_bounds_check_build():
    from paper_1607_03062_gb300 import build
    lib = build.build(bounds_check=True)
    env = dict(os.environ, DSP_LIBRARY=lib)
    out = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "gpu",
         os.path.join(ROOT, "tests", "test_gpu_parity.py"),
         os.path.join(ROOT, "tests", "test_time_parallel.py"),
         os.path.join(ROOT, "tests", "test_serving.py"),
         "-k", "not full_size and not timeout"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout
