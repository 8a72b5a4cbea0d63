"""D2Q9 variant of the step (the same recursion on D1Q3 x D1Q3) against the
FP64 D2Q9 oracle, through the C ABI (lattice TSLB_D2Q9, dims = (nx, ny, 1)).

Tolerances as for D3Q27: 2e-6 after one step on random moments (FP32
rounding and summation order only), 1e-5 for u and Pi^neq after 200
Taylor-Green steps (2e-5 for rho - 1, a difference of cancelling fluxes),
and the forced bounce-back channel at the bench relaxation time.  The full
bench-size channel (8192 x 2050) is compared at every node after two steps.
"""
import math

import numpy as np
import pytest

from hypothesis import HealthCheck, given, settings
from hypothesis import strategies as st

import oracle
import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu
FIELDS = ["drho", "ux", "uy", "pxx", "pyy", "pxy"]


def _to2d(rho, u, pi):
    return rho, np.stack([u[0], u[1]]), np.stack([pi[0], pi[1], pi[3]])


def _stack2(rho, u2, pi3):
    return np.concatenate([(rho - 1.0)[None], u2, pi3])


def _run(dims, tau, state, nsteps, bc=(0, 0, 0, 0, 0, 0), force=(0.0, 0.0, 0.0), zero_fields=()):
    """Relative L2 error per field; fields in zero_fields (analytically zero)
    are measured absolutely against the norm of the non-zero field of the same
    order (u for u, Pi_xx for Pi)."""
    nx, ny, _ = dims
    o = oracle.OracleSim2D((nx, ny), tau, force=force[:2], bc=bc[:4])
    o.init_moments(*_to2d(*state))
    o.step(nsteps)
    ref = _stack2(*o.get_moments())
    s = T.Solver(dims, tau, force=force, bc=bc, lattice=T.TSLB_D2Q9)
    s.init_moments(*state)
    s.step(nsteps)
    r, u, p = s.get_moments()
    s.close()
    got = _stack2(*_to2d(r, u, p))
    assert np.abs(u[2]).max() == 0 and np.abs(p[[2, 4, 5]]).max() == 0
    inner = np.ones((ny, nx), bool)
    if bc[2]:
        inner[[0, ny - 1], :] = False
    m = inner.reshape(-1)
    errs = {}
    for k, name in enumerate(FIELDS):
        d = got[k][m] - ref[k][m]
        nrm = np.linalg.norm(ref[k][m])
        if name in zero_fields:
            nrm = np.linalg.norm(ref[1 if name in ("ux", "uy") else 3][m])
        errs[name] = float(np.linalg.norm(d) / nrm) if nrm > 0 else float(np.abs(d).max())
    return errs


def _random3(dims, seed, drho=0.01, du=0.05, dpi=1e-3):
    rho, u, pi = W.random_state(dims, seed=seed, drho=drho, du=du, dpi=dpi)
    u = u.copy()
    pi = pi.copy()
    u[2] = 0.0
    pi[[2, 4, 5]] = 0.0
    return rho, u, pi


@pytest.mark.parametrize("dims", [(40, 37, 1), (7, 5, 1), (64, 200, 1)], ids=["ragged-x", "small", "tall"])
def test_one_step_random_periodic(cuda_ok, dims):
    errs = _run(dims, 0.6, _random3(dims, 41), 1)
    assert max(errs.values()) <= 2e-6, errs


def test_taylor_green_200_steps(cuda_ok):
    n, u0, tau = 64, 0.05, 0.6
    k = 2 * math.pi / n
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    x, y = x.reshape(-1), y.reshape(-1)
    N = n * n
    u = np.zeros((3, N))
    u[0] = -u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = u0 * np.sin(k * x) * np.cos(k * y)
    d = u0 * k * np.sin(k * x) * np.sin(k * y)
    pi = np.zeros((6, N))
    pi[0] = -2.0 / 3.0 * tau * d
    pi[1] = 2.0 / 3.0 * tau * d
    errs = _run((n, n, 1), tau, (np.ones(N), u, pi), 200, zero_fields=("pxy",))
    assert errs["drho"] <= 2e-5, errs
    assert max(v for kk, v in errs.items() if kk != "drho") <= 1e-5, errs


@pytest.mark.parametrize("dims", [(33, 20, 1), (61, 170, 1), (12, 4, 1)], ids=["one-chunk", "ragged-chunks", "two-rows"])
def test_bounceback_channel(cuda_ok, dims):
    bc = (0, 0, 1, 1, 0, 0)
    errs = _run(dims, 0.6, _random3(dims, 42), 5, bc=bc, force=(2e-5, -1e-5, 0.0))
    assert max(errs.values()) <= 3e-6, errs


def test_forced_channel_bench_tau(cuda_ok):
    prm = W.channel2d_params(nx=96, ny=66)
    errs = _run(prm["dims"], prm["tau"], W.channel2d_state(prm, seed=2), 30, bc=prm["bc"], force=prm["force"])
    assert errs["ux"] <= 1e-5, errs
    assert max(errs.values()) <= 1e-4, errs


def test_channel_full_size(cuda_ok):
    """The bench workload (8192 x 2050, 16.78 M interior nodes), every node, two steps."""
    prm = W.channel2d_params()
    errs = _run(prm["dims"], prm["tau"], W.channel2d_state(prm, seed=1), 2, bc=prm["bc"], force=prm["force"])
    assert errs["ux"] <= 3e-6 and errs["uy"] <= 3e-6, errs
    assert max(errs.values()) <= 2e-5, errs


def test_d2q9_rejections(cuda_ok):
    s = T.Solver((16, 8, 1), 0.6, lattice=T.TSLB_D2Q9)
    with pytest.raises(T.TslbError) as ei:
        s.set_force_field(np.zeros((3, 128), np.float32))
    assert ei.value.code == T.TSLB_ERR_UNSUPPORTED
    s.close()



@settings(max_examples=60, deadline=None,
          suppress_health_check=[HealthCheck.too_slow, HealthCheck.function_scoped_fixture])
@given(nx=st.integers(3, 100), ny=st.integers(4, 300), walls=st.booleans(), tau=st.floats(0.55, 1.5),
       seed=st.integers(0, 10 ** 6), F=st.tuples(st.floats(-2e-5, 2e-5), st.floats(-2e-5, 2e-5)))
def test_random_boxes_two_steps(cuda_ok, nx, ny, walls, tau, seed, F):
    """Random box sizes (ragged against the 30-column warps and the y chunks of
    the one-wave grid), periodic or bounce-back y faces, tau, force and seed:
    two steps from random moments within 4e-6 per field (twice the one-step
    bound)."""
    dims = (nx, ny, 1)
    bc = (0, 0, 1, 1, 0, 0) if walls else (0,) * 6
    errs = _run(dims, tau, _random3(dims, seed), 2, bc=bc, force=(F[0], F[1], 0.0))
    assert max(errs.values()) <= 4e-6, (errs, dims, walls, tau)
