"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

Builds liboracle_san.so (ORACLE_SANITIZE=1: g++ -fsanitize=address,undefined)
and drives every oracle entry point on small boxes in a child process with
the ASan runtime preloaded: the lattice and Hermite helpers, Philox and both
inflow noises, every face type, the sponge layer, Guo forcing with a force
field, the population read-out, the complex-step run and the D2Q9 oracle.  An
invalid memory access or undefined behaviour ends the child with an error.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import oracle
from paper_2401_17074_b300 import workloads as W

oracle.lattice()
rng = np.random.default_rng(0)
u = np.array([0.03, -0.02, 0.01])
oracle.feq3(1.01, u)
oracle.fneq3(1e-3 * rng.standard_normal(6), u)
oracle.post_collision(1.0, u, 1e-3 * rng.standard_normal(6), 1.2, (1e-5, 0.0, 0.0))
oracle.moments(oracle.feq3(1.0, u))
oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
oracle.inflow_noise(3, 1, 2, 3)
oracle.inflow_noise_gauss(3, 1, 2, 3)

def run(dims, bc, steps=2, **kw):
    s = oracle.OracleSim(dims, 0.6, bc=bc, **kw)
    s.init_moments(*W.random_state(dims, seed=1, drho=0.002, du=0.01, dpi=1e-4))
    s.step(steps)
    s.get_moments()
    return s

run((5, 6, 7), (0,) * 6)
run((6, 7, 5), (0, 0, 1, 1, 0, 0), force=(1e-5, 0.0, 0.0))
run((6, 7, 5), (0, 0, 5, 5, 0, 0), force=(1e-5, 0.0, 0.0))
run((7, 6, 5), (2, 2, 2, 2, 0, 0))
run((8, 8, 9), (2, 2, 2, 2, 3, 4), inflow=dict(center2=(4, 4), diameter=4, u_jet=0.05, noise_amp=0.01, seed=3))
run((8, 8, 12), (0, 0, 0, 0, 3, 4), inflow=dict(center2=(4, 4), diameter=4, u_jet=0.05, noise_amp=0.01, seed=3,
                                                 noise="gaussian"), sponge=(4, 100.0))
g = oracle.OracleSim((5, 6, 4), 0.7, forcing="guo", bc=(0, 0, 1, 1, 0, 0))
g.set_force_field(1e-5 * rng.standard_normal((3, 120)))
g.init_moments(*W.random_state((5, 6, 4), seed=2))
g.step(2)
g.get_moments()
g.get_populations()
dims = (4, 4, 4)
st = W.random_state(dims, seed=3)
oracle.complex_step_energy(dims, 0.7, (0,) * 6, st[0], st[1], st[2], np.zeros((3, 64)),
                           1e-30 * rng.standard_normal((3, 64)), 2)
for bc in ((0, 0, 0, 0), (0, 0, 1, 1)):
    s2 = oracle.OracleSim2D((7, 6), 0.6, force=(1e-5, 0.0), bc=bc)
    s2.init_moments(np.ones(42), 0.01 * rng.standard_normal((2, 42)), 1e-4 * rng.standard_normal((3, 42)))
    s2.step(3)
    s2.get_moments()
print("sanitized oracle ok")
"""


def test_oracle_under_asan_and_ubsan():
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    env = dict(os.environ, ORACLE_SANITIZE="1", LD_PRELOAD=asan, OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "sanitized oracle ok" in r.stdout
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
