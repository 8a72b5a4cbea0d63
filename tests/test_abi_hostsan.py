"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer.

Builds libtslb_hostsan.so (the host code compiled with -fsanitize=address and
-fsanitize=undefined; device code unchanged) and runs the CPU tests of the C
ABI against it in a child process with the ASan runtime preloaded (TSLB_HOSTSAN=1):
argument and option validation of tslb_create, the option defaults, the
handle-free error paths.  An invalid access or undefined behaviour in that host
code ends the child with an error.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_abi_host_paths_under_asan_and_ubsan():
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    sys.path.insert(0, ROOT)
    from paper_2401_17074_b300 import build as B
    B.build_hostsan()
    env = dict(os.environ, TSLB_HOSTSAN="1", LD_PRELOAD=asan,
               # the CUDA runtime maps memory in ASan's shadow gap
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    probe = ("import paper_2401_17074_b300 as T; T.load(build_if_missing=False); "
             "assert T.lib_path().endswith('libtslb_hostsan.so'), T.lib_path()")
    r = subprocess.run([sys.executable, "-c", probe], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "tests/test_abi_cpu.py"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
