"""The CUDA path against closed forms of the physics, without the oracle.

- Steady Poiseuille flow between walls: the body force g balances viscosity,
  nu = cs^2 (tau - 1/2), and the velocity is the parabola
  u(y) = g / (2 nu) (y - y0)(y1 - y).  Halfway bounce-back puts the walls half
  a node outside the last fluid rows (y0 = 1/2, y1 = ny - 3/2); the thread-safe
  NEE walls of Sec. 2.3 sit on the nodes y = 0 and y = ny - 1.  Regularised
  walls carry a tau-dependent slip of O(1/H^2) relative, so the pin is second
  order convergence over H = 8, 16, 32 (from rest, 6 H^2 / nu steps, which
  damps the slowest transient by e^-59).
- Taylor-Green vortex: the amplitude decays as exp(-2 nu k^2 t); the fitted
  viscosity is within 1 % of cs^2 (tau - 1/2) (the lattice's O(k^2) error at
  k = 2 pi / 32 is below that).
- Checkpoint / resume through the public API: moments read back and loaded
  into a new solver continue the run bit for bit (FP32 and BF16: the decode
  and re-encode of a stored value return it exactly).
"""
import math

import numpy as np
import pytest

import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


def _poiseuille_error(H, wall, tau=0.8, lattice=None, kernel=T.KERNEL_AUTO):
    nu = CS2 * (tau - 0.5)
    g = 0.01 * 8 * nu / H ** 2  # centreline velocity about 0.01
    if wall == "bounce-back":
        ny, bc, y0, y1 = H + 2, 1, 0.5, H + 0.5
    else:
        ny, bc, y0, y1 = H + 1, T.NEE_WALL, 0.0, float(H)
    dims = (3, ny, 1) if lattice == T.TSLB_D2Q9 else (3, ny, 3)
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, tau, force=(g, 0.0, 0.0), bc=(0, 0, bc, bc, 0, 0), lattice=lattice, kernel=kernel)
    s.init_moments(np.ones(N), np.zeros((3, N)), np.zeros((6, N)))
    s.step(int(6 * H * H / nu))
    _, u, _ = s.get_moments()
    s.close()
    y = np.arange(ny, dtype=float)
    prof = u[0].reshape(dims[2], ny, dims[0]).mean(axis=(0, 2))
    fluid = slice(1, ny - 1)
    exact = g / (2 * nu) * (y - y0) * (y1 - y)
    e = prof[fluid] - exact[fluid]
    return float(np.sqrt(np.mean(e ** 2)) / np.sqrt(np.mean(exact[fluid] ** 2)))


@pytest.mark.parametrize("case", [("bounce-back", None), ("nee", None), ("bounce-back", "d2q9")],
                         ids=["bounce-back", "nee-walls", "d2q9-bounce-back"])
def test_poiseuille_second_order(cuda_ok, case):
    wall, lat = case
    lattice = T.TSLB_D2Q9 if lat == "d2q9" else None
    e8, e16, e32 = (_poiseuille_error(H, wall, lattice=lattice) for H in (8, 16, 32))
    assert e8 < 0.06, (e8, e16, e32)
    assert math.log2(e8 / e16) > 1.8 and math.log2(e16 / e32) > 1.8, (e8, e16, e32)


def _tgv_amplitude(u, dims):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = 2 * math.pi / nx
    mode = (-np.cos(k * x) * np.sin(k * y)).reshape(-1)
    return float(np.dot(u[0], mode) / np.dot(mode, mode))


@pytest.mark.parametrize("lattice", [None, T.TSLB_D2Q9], ids=["d3q27", "d2q9"])
def test_taylor_green_viscosity(cuda_ok, lattice):
    n, tau, steps = 32, 0.6, 400
    dims, state = W.taylor_green(n=n, u0=0.05, tau=tau)
    if lattice == T.TSLB_D2Q9:  # one z layer of the same field
        N2 = n * n
        dims = (n, n, 1)
        state = (state[0][:N2], state[1][:, :N2], state[2][:, :N2])
    s = T.Solver(dims, tau, lattice=lattice)
    s.init_moments(*state)
    a0 = _tgv_amplitude(s.get_moments()[1], dims)
    s.step(steps)
    a1 = _tgv_amplitude(s.get_moments()[1], dims)
    s.close()
    k = 2 * math.pi / n
    nu_fit = -math.log(a1 / a0) / (2 * k * k * steps)
    nu = CS2 * (tau - 0.5)
    assert abs(nu_fit - nu) <= 0.01 * nu, (nu_fit, nu)


@pytest.mark.parametrize("prec", [T.FP32, T.BF16], ids=["fp32", "bf16"])
def test_resume_from_saved_moments(cuda_ok, prec):
    prm = W.channel_params(nx=40, ny=34, nz=20)
    state = W.channel_state(prm, seed=3)
    kw = dict(force=prm["force"], bc=prm["bc"], precision=prec, u_ref=0.05, pi_ref=W.pi_reference(state))
    a = T.Solver(prm["dims"], prm["tau"], **kw)
    a.init_moments(*state)
    a.step(7)
    saved = a.get_moments()
    a.step(5)
    ref = a.get_moments()
    a.close()
    b = T.Solver(prm["dims"], prm["tau"], **kw)
    b.init_moments(*saved)
    b.step(5)
    got = b.get_moments()
    b.close()
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
