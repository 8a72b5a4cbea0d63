"""The index-checked build (libtslb_checked.so, TSLB_CHECKED=1).

Every kernel of that build tests its global-memory indices, and the step
kernel its shared-memory exchange offsets, and records an index out of range
in the device status word instead of faulting (the calls then fail with
TSLB_ERR_CUDA).  The GPU parity suites run against it in a child process: they
must pass as they do with the product library, so no index of any tested
configuration leaves its array.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_under_the_checked_build(cuda_ok):
    env = dict(os.environ, TSLB_CHECKED="1")
    probe = ("import paper_2401_17074_b300 as T; T.load(build_if_missing=False); "
             "assert T.lib_path().endswith('libtslb_checked.so'), T.lib_path()")
    r = subprocess.run([sys.executable, "-c", probe], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    suites = ["tests/test_parity_gpu.py", "tests/test_d2q9_gpu.py", "tests/test_rounding_gpu.py",
              "tests/test_physics_gpu.py", "tests/test_adjoint_gpu.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "-k", "not complex_step_128"] + suites,
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
