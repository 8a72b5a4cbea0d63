"""Oracle invariants over random shapes, relaxation times, states and forces
(property-based, hypothesis).

- Periodic box: the streaming of Eq. pushLB moves populations without loss,
  and the collision keeps mass and momentum (Sec. 2.1) while the Luo term of
  Sec. 3.1 adds rho F: after n steps, sum rho is unchanged and sum rho u has
  grown by n F sum rho, to FP64 round-off.
- The rest state (rho = 1, u = 0, Pi = 0, no force) stays at rest exactly, with
  any of the wall types on the y faces.
- The D2Q9 oracle keeps the same balances in two dimensions.
"""
import numpy as np
from hypothesis import HealthCheck, given, settings
from hypothesis import strategies as st

import oracle
from paper_2401_17074_b300 import workloads as W

SETTINGS = settings(max_examples=100, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@SETTINGS
@given(nx=st.integers(3, 7), ny=st.integers(3, 7), nz=st.integers(3, 7), tau=st.floats(0.52, 1.8),
       seed=st.integers(0, 10 ** 6), steps=st.integers(1, 4),
       F=st.tuples(*[st.floats(-1e-4, 1e-4)] * 3))
def test_periodic_mass_and_momentum_balance(nx, ny, nz, tau, seed, steps, F):
    dims = (nx, ny, nz)
    rho, u, pi = W.random_state(dims, seed=seed, drho=0.01, du=0.03, dpi=1e-4)
    s = oracle.OracleSim(dims, tau, force=F)
    s.init_moments(rho, u, pi)
    r0, u0, _ = s.get_moments()
    M = r0.sum()
    P0 = (r0 * u0).sum(axis=1)
    s.step(steps)
    r1, u1, _ = s.get_moments()
    assert abs(r1.sum() - M) <= 1e-12 * M
    P1 = (r1 * u1).sum(axis=1)
    expect = P0 + steps * np.asarray(F) * M
    assert np.all(np.abs(P1 - expect) <= 1e-12 * M), (P1, expect)


@SETTINGS
@given(nx=st.integers(3, 6), ny=st.integers(4, 8), nz=st.integers(3, 6), tau=st.floats(0.52, 1.8),
       wall=st.sampled_from([oracle.BOUNCEBACK, oracle.FREESLIP, oracle.NEE_WALL]), steps=st.integers(1, 4))
def test_rest_state_stays_at_rest(nx, ny, nz, tau, wall, steps):
    dims = (nx, ny, nz)
    N = nx * ny * nz
    s = oracle.OracleSim(dims, tau, bc=(0, 0, wall, wall, 0, 0))
    s.init_moments(np.ones(N), np.zeros((3, N)), np.zeros((6, N)))
    s.step(steps)
    r, u, p = s.get_moments()
    interior = np.zeros((nz, ny, nx), bool)
    interior[:, 1:ny - 1, :] = True
    interior = interior.reshape(-1)
    assert np.abs(r[interior] - 1.0).max() <= 1e-14
    assert np.abs(u[:, interior]).max() <= 1e-14 and np.abs(p[:, interior]).max() <= 1e-14


@SETTINGS
@given(nx=st.integers(3, 9), ny=st.integers(3, 9), tau=st.floats(0.52, 1.8), seed=st.integers(0, 10 ** 6),
       steps=st.integers(1, 4), F=st.tuples(*[st.floats(-1e-4, 1e-4)] * 2))
def test_d2q9_periodic_mass_and_momentum_balance(nx, ny, tau, seed, steps, F):
    N = nx * ny
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.01 * rng.uniform(-1, 1, N)
    u = 0.03 * rng.uniform(-1, 1, (2, N))
    pi = 1e-4 * rng.uniform(-1, 1, (3, N))
    s = oracle.OracleSim2D((nx, ny), tau, force=F)
    s.init_moments(rho, u, pi)
    r0, u0, _ = s.get_moments()
    M = r0.sum()
    P0 = (r0 * u0).sum(axis=1)
    s.step(steps)
    r1, u1, _ = s.get_moments()
    assert abs(r1.sum() - M) <= 1e-12 * M
    expect = P0 + steps * np.asarray(F) * M
    assert np.all(np.abs((r1 * u1).sum(axis=1) - expect) <= 1e-12 * M)
