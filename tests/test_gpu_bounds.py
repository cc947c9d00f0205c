"""Run the GPU parity tests against the bounds-checked build of the library
(libmorse_checked.so, MORSE_LIB=checked): every texel index the search
computes is range-checked in device code; a violation sets an error bit,
skips the access and makes the call fail on the host.  No trap, no fault."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_bounds_checks():
    lib = os.path.join(ROOT, "paper_1511_01157_gb300", "libmorse_checked.so")
    if not os.path.exists(lib):
        pytest.fail("libmorse_checked.so not built (run build())")
    env = dict(os.environ, MORSE_LIB="checked")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
         "-p", "no:cacheprovider", os.path.join(ROOT, "tests",
                                               "test_gpu_parity.py")],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
