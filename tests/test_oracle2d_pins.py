"""Pins of the D2Q9 oracle (oracle/tslb_oracle2d.cpp) against what the paper
and the mathematics fix, independently of the oracle's own formulas.

Lattice: weights 4/9, 1/9, 1/36 with isotropic moments up to fourth order.
Equilibrium (Eq. eqts) and regularised non-equilibrium (Eq. noneqts): their
moments up to the lattice-supported third order.  Dynamics: rest state,
uniform flow, conservation, Luo forcing (Sec. 3.1), the viscosity
nu = cs^2 (tau - 1/2) through Taylor-Green decay, and second-order
Poiseuille flow between halfway bounce-back walls.
"""
import math

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat():
    return oracle.lattice2d()


def test_lattice_weights_and_isotropy(lat):
    c, w = lat
    assert abs(w.sum() - 1.0) < 1e-15
    classes = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    for i in range(9):
        assert abs(w[i] - classes[int(np.abs(c[i]).sum())]) < 1e-15
    d = np.eye(2)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.abs(m2 - CS2 * d).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(m4 - iso).max() < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15


def test_feq3_moments(lat):
    c, _ = lat
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(2)
        f = oracle.feq3_2d(rho, u)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(f @ c - rho * u).max() < 1e-14
        m2 = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.abs(m2 - rho * np.outer(u, u) - rho * CS2 * np.eye(2)).max() < 1e-14
        # third moments the lattice supports: Q_xyy and Q_xxy
        qxyy = np.sum(f * c[:, 0] * c[:, 1] ** 2)
        qxxy = np.sum(f * c[:, 0] ** 2 * c[:, 1])
        assert abs(qxyy - rho * (u[0] * u[1] ** 2 + CS2 * u[0])) < 1e-14
        assert abs(qxxy - rho * (u[0] ** 2 * u[1] + CS2 * u[1])) < 1e-14


def test_fneq3_projection(lat):
    c, _ = lat
    rng = np.random.default_rng(2)
    for _ in range(20):
        u = 0.1 * rng.standard_normal(2)
        p3 = 1e-3 * rng.standard_normal(3)
        P = np.array([[p3[0], p3[2]], [p3[2], p3[1]]])
        f = oracle.fneq3_2d(p3, u)
        assert abs(f.sum()) < 1e-17
        assert np.abs(f @ c).max() < 1e-17
        assert np.abs(np.einsum("i,ia,ib->ab", f, c, c) - P).max() < 1e-17
        # third-order coefficient a3_abb = u_a Pi_bb + 2 u_b Pi_ab
        assert abs(np.sum(f * c[:, 0] * c[:, 1] ** 2) - (u[0] * P[1, 1] + 2 * u[1] * P[0, 1])) < 1e-17
        assert abs(np.sum(f * c[:, 0] ** 2 * c[:, 1]) - (u[1] * P[0, 0] + 2 * u[0] * P[0, 1])) < 1e-17


def _random_state(dims, seed, drho=0.01, du=0.05, dpi=1e-3):
    rng = np.random.default_rng(seed)
    N = dims[0] * dims[1]
    return 1 + drho * rng.uniform(-1, 1, N), du * rng.uniform(-1, 1, (2, N)), dpi * rng.uniform(-1, 1, (3, N))


def test_rest_and_uniform_flow():
    dims = (7, 5)
    N = 35
    s = oracle.OracleSim2D(dims, 0.7)
    s.init_moments(np.ones(N), np.zeros((2, N)))
    s.step(10)
    r, u, p = s.get_moments()
    assert np.abs(r - 1).max() < 1e-14 and np.abs(u).max() < 1e-15 and np.abs(p).max() < 1e-15
    U = np.array([0.03, -0.02])
    s = oracle.OracleSim2D(dims, 0.6)
    s.init_moments(np.ones(N) * 1.01, np.tile(U[:, None], (1, N)))
    s.step(10)
    r, u, p = s.get_moments()
    assert np.abs(r - 1.01).max() < 1e-13 and np.abs(u - U[:, None]).max() < 1e-14 and np.abs(p).max() < 1e-14


def test_conservation_and_forcing():
    dims = (6, 7)
    rho, u, pi = _random_state(dims, 3)
    s = oracle.OracleSim2D(dims, 0.58)
    s.init_moments(rho, u, pi)
    m0, p0 = rho.sum(), (rho[None] * u).sum(1)
    s.step(50)
    r, uu, _ = s.get_moments()
    assert abs(r.sum() - m0) / m0 < 1e-13
    assert np.abs((r[None] * uu).sum(1) - p0).max() < 1e-13 * m0
    F = np.array([2e-6, -3e-6])
    s = oracle.OracleSim2D(dims, 0.7, force=F)
    s.init_moments(rho, u, pi)
    s.step(20)
    r, uu, _ = s.get_moments()
    assert np.abs((r[None] * uu).sum(1) - (p0 + 20 * F * m0)).max() < 1e-13


def test_taylor_green_decay():
    """2-D Taylor-Green vortex: amplitude ~ exp(-2 nu k^2 t), nu = cs^2 (tau - 1/2)."""
    n, u0, tau = 32, 0.02, 0.6
    k = 2 * math.pi / n
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    x, y = x.reshape(-1), y.reshape(-1)
    u = np.array([-u0 * np.cos(k * x) * np.sin(k * y), u0 * np.sin(k * x) * np.cos(k * y)])
    # Pi^neq from the strain: -rho cs^2 tau (d_a u_b + d_b u_a)
    dxux = u0 * k * np.sin(k * x) * np.sin(k * y)
    sxy = 0.0 * x  # d_y u_x + d_x u_y = -u0 k cos cos + u0 k cos cos = 0
    pi = -CS2 * tau * np.array([2 * dxux, -2 * dxux, sxy])
    s = oracle.OracleSim2D((n, n), tau)
    s.init_moments(np.ones(n * n), u, pi)
    ts, amps = [], []
    for _ in range(5):
        s.step(40)
        _, uu, _ = s.get_moments()
        ts.append((len(ts) + 1) * 40)
        amps.append(np.sqrt(np.mean(uu[0] ** 2 + uu[1] ** 2)))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    nu = CS2 * (tau - 0.5)
    assert abs(rate / (2 * nu * k * k) - 1) < 0.01


def _poiseuille_error(H, tau=0.8, g=1e-6):
    ny = H + 2
    dims = (3, ny)
    N = 3 * ny
    nu = CS2 * (tau - 0.5)
    y = np.repeat(np.arange(ny, dtype=float), 3)
    y0, y1 = 0.5, ny - 1.5
    exact = g / (2 * nu) * (y - y0) * (y1 - y)
    fluid = (y >= 1) & (y <= ny - 2)
    u = np.zeros((2, N))
    u[0] = np.where(fluid, exact, 0.0)
    pi = np.zeros((3, N))
    pi[2] = np.where(fluid, -CS2 * tau * g / (2 * nu) * (y1 + y0 - 2 * y), 0.0)
    s = oracle.OracleSim2D(dims, tau, force=(g, 0.0), bc=(0, 0, 1, 1))
    s.init_moments(np.ones(N), u, pi)
    s.step(int(3 * H * H / nu))
    _, uu, _ = s.get_moments()
    e = uu[0][fluid] - exact[fluid]
    return np.sqrt(np.mean(e ** 2)) / np.sqrt(np.mean(exact[fluid] ** 2))


def test_poiseuille_bounceback_second_order():
    e8, e16, e32 = (_poiseuille_error(H) for H in (8, 16, 32))
    assert e8 < 0.05
    assert math.log2(e8 / e16) > 1.8 and math.log2(e16 / e32) > 1.8
