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


@pytest.mark.parametrize("kernel", [T.KERNEL_FACTORED, T.KERNEL_DIRECT], ids=["factored", "direct"])
def test_wall_shear_diagnostic_poiseuille(cuda_ok, kernel):
    """The wall-shear diagnostic against the closed form: in steady Poiseuille
    flow between halfway bounce-back walls the shear stress is linear,
    sigma_xy(y) = rho g (y_c - y), so at the wall-adjacent nodes (half a node
    from the walls) the diagnostic -(1 - omega/2) Pi_xy must read
    rho g (H - 1/2) with H the half-width.  The regularised scheme reproduces
    the linear stress exactly (the oracle: 1e-12); the bound 1e-4 covers the
    FP32 storage of Pi^neq and the remaining transient (8 H^2 / nu steps)."""
    H, tau = 8, 0.8
    nu = CS2 * (tau - 0.5)
    g = 0.01 * 8 * nu / (2 * H) ** 2
    ny = 2 * H + 2
    dims = (4, ny, 4)
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, tau, force=(g, 0.0, 0.0), bc=(0, 0, 1, 1, 0, 0), kernel=kernel)
    s.init_moments(np.ones(N), np.zeros((3, N)), np.zeros((6, N)))
    s.step(int(8 * (2 * H) ** 2 / nu))
    d, code = s.diagnostics()
    rho, _, _ = s.get_moments()
    s.close()
    assert code == T.TSLB_OK
    fluid = ((np.arange(N) // dims[0]) % ny >= 1) & ((np.arange(N) // dims[0]) % ny <= ny - 2)
    want = float(rho[fluid].mean()) * g * (H - 0.5)
    assert abs(d["wall_shear"] / want - 1) < 1e-4, (d["wall_shear"], want)


def test_wall_shear_diagnostic_numpy_sum(cuda_ok):
    """On a walled box in a non-trivial state (random moments, eleven steps),
    tslb_diagnostics' FP64 wall shear equals the mean of -(1 - omega/2) Pi_xy
    over the nodes of y = 1 and of +(1 - omega/2) Pi_xy over y = ny - 2,
    summed in numpy from the moments read back (1e-12 relative); with NEE walls
    the same rows count."""
    for bcy in (1, T.NEE_WALL):
        dims, tau = (13, 9, 7), 0.57
        N = dims[0] * dims[1] * dims[2]
        s = T.Solver(dims, tau, force=(1e-5, 0.0, 0.0), bc=(0, 0, bcy, bcy, 0, 0))
        s.init_moments(*W.random_state(dims, seed=71, drho=0.005, du=0.02, dpi=1e-3))
        s.step(11)
        d, code = s.diagnostics()
        _, _, pi = s.get_moments()
        s.close()
        assert code == T.TSLB_OK
        y = (np.arange(N) // dims[0]) % dims[1]
        sc = 1.0 - 0.5 / tau
        want = (np.sum(-sc * pi[3][y == 1]) + np.sum(sc * pi[3][y == dims[1] - 2])) / (2 * dims[0] * dims[2])
        assert abs(d["wall_shear"] - want) <= 1e-12 * abs(want), (bcy, d["wall_shear"], want)
