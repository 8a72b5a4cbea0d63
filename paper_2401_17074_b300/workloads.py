"""Seeded synthetic inputs for the TSLB workloads (initial moments and set-ups).

This module only builds initial conditions and problem parameters; it holds
none of the step's arithmetic and is shared by the CUDA path, the oracle
tests and the benchmark.  Arrays use the C ABI layout: full lattice,
x fastest, rho [N], u [3][N], pi [6][N] (xx, yy, zz, xy, xz, yz).

Where an initial Pi^neq is wanted it is the Navier-Stokes estimate of the
non-equilibrium momentum flux of the initial velocity field,
Pi_ab = -rho cs^2 tau (d_a u_b + d_b u_a) (Chapman-Enskog; arXiv 2401.17074
quotes the same relation for a^2_neq in Sec. 2.2), evaluated from the
analytic (or spectral) velocity gradient of the prescribed field.

The workloads stand in for the paper's flows (Sec. 3): there are no datasets;
every input is generated here from a seed.
"""
import math

import numpy as np

CS2 = 1.0 / 3.0
PERIODIC, BOUNCEBACK, FREESLIP, INFLOW, OUTFLOW, NEE_WALL = 0, 1, 2, 3, 4, 5


def _coords(dims):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def _pack(rho, u, pi):
    return (np.ascontiguousarray(rho, dtype=np.float64),
            np.ascontiguousarray(np.stack(u), dtype=np.float64),
            np.ascontiguousarray(np.stack(pi), dtype=np.float64))


def random_state(dims, seed, drho=0.01, du=0.05, dpi=1e-3):
    """Uniform random moments: rho = 1 + drho xi, u = du xi, Pi = dpi xi (xi ~ U(-1,1))."""
    rng = np.random.default_rng(seed)
    N = dims[0] * dims[1] * dims[2]
    rho = 1.0 + drho * rng.uniform(-1, 1, N)
    u = du * rng.uniform(-1, 1, (3, N))
    pi = dpi * rng.uniform(-1, 1, (6, N))
    return _pack(rho, list(u), list(pi))


def pi_reference(state, headroom=2.0, floor=1e-6):
    """Scale of Pi^neq for 16-bit storage: headroom x the largest |Pi^neq| of a state."""
    return max(floor, headroom * float(np.abs(state[2]).max()))


def rest_state(dims):
    N = dims[0] * dims[1] * dims[2]
    return _pack(np.ones(N), [np.zeros(N)] * 3, [np.zeros(N)] * 6)


def taylor_green(n=32, u0=0.05, tau=0.6, with_pi=True):
    """2-D Taylor-Green vortex on an n^3 periodic box (config: 32^3, u0=0.05, tau=0.6).

    u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), u_z = 0, k = 2 pi / n, rho = 1.
    Its amplitude decays as exp(-2 nu k^2 t) with nu = cs^2 (tau - 1/2).
    """
    dims = (n, n, n)
    x, y, z = _coords(dims)
    k = 2.0 * math.pi / n
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    uz = np.zeros_like(x)
    rho = np.ones_like(x)
    zero = np.zeros_like(x)
    pi = [zero] * 6
    if with_pi:
        dxux = u0 * k * np.sin(k * x) * np.sin(k * y)
        dyuy = -u0 * k * np.sin(k * x) * np.sin(k * y)
        dyux = -u0 * k * np.cos(k * x) * np.cos(k * y)
        dxuy = u0 * k * np.cos(k * x) * np.cos(k * y)
        c = -rho * CS2 * tau
        pi = [c * 2 * dxux, c * 2 * dyuy, zero, c * (dyux + dxuy), zero, zero]
    return dims, _pack(rho, [ux, uy, uz], pi)


def shear_wave(dims, amp, tau, axis_u=0, axis_k=1, mode=1):
    """u_a = amp sin(k y) on a periodic box, k = 2 pi mode / n_k; decays as exp(-nu k^2 t)."""
    x, y, z = _coords(dims)
    coords = (x, y, z)
    k = 2.0 * math.pi * mode / dims[axis_k]
    s = coords[axis_k]
    u = [np.zeros_like(x) for _ in range(3)]
    u[axis_u] = amp * np.sin(k * s)
    rho = np.ones_like(x)
    pi = [np.zeros_like(x) for _ in range(6)]
    # Pi_ab for the single shear component d u_a / d s
    grad = amp * k * np.cos(k * s)
    off = {(0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    if axis_u != axis_k:
        pi[off[(axis_u, axis_k)]] = -rho * CS2 * tau * grad
    return _pack(rho, u, pi)


# ---- turbulent channel (Sec. 3.1 shape; benchmark grid 512 x 130 x 256) -----

def channel_params(nx=512, ny=130, nz=256, u_tau=0.0035, tau=0.503, re_tau=180.0):
    """Walls at y = 0 and y = ny-1 (solid layers, halfway bounce-back), H = (ny-2)/2.

    Body force g = u_tau^2 / H along x (u_tau = sqrt(g H), Sec. 3.1).
    """
    H = (ny - 2) / 2.0
    g = u_tau * u_tau / H
    return dict(dims=(nx, ny, nz), tau=tau, force=(g, 0.0, 0.0),
                bc=(PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK, PERIODIC, PERIODIC),
                H=H, u_tau=u_tau, re_tau=re_tau)


def channel_state(prm, seed=1, noise=0.02):
    """Laminar parabola scaled to the log-law centreline velocity plus seeded noise.

    U_c = u_tau (ln(Re_tau)/0.41 + 5) (log-law constants quoted in Sec. 3.1);
    u_x = U_c (1 - ((y - y_c)/H)^2) with walls at y = 1/2 and y = ny - 3/2;
    every velocity component gets noise * U_c * xi, xi ~ U(-1, 1), seeded.
    Pi^neq from the parabola's shear; boundary-layer nodes are at rest.
    """
    nx, ny, nz = prm["dims"]
    H, tau = prm["H"], prm["tau"]
    Uc = prm["u_tau"] * (math.log(prm["re_tau"]) / 0.41 + 5.0)
    yc = 0.5 + H  # midway between the walls at 1/2 and ny - 3/2
    N = nx * ny * nz
    rng = np.random.default_rng(seed)
    yv = np.arange(ny, dtype=np.float64)
    prof = Uc * (1.0 - ((yv - yc) / H) ** 2)
    dprof = -2.0 * Uc * (yv - yc) / (H * H)
    fluid = (yv >= 1) & (yv <= ny - 2)
    prof[~fluid] = 0.0
    dprof[~fluid] = 0.0
    shape = (nz, ny, nx)
    ux = np.broadcast_to(prof[None, :, None], shape).reshape(-1).copy()
    pxy = np.broadcast_to((-CS2 * tau * dprof)[None, :, None], shape).reshape(-1).copy()
    u = [ux, np.zeros(N), np.zeros(N)]
    for a in range(3):
        u[a] += noise * Uc * rng.uniform(-1.0, 1.0, N)
    mask = np.broadcast_to(fluid[None, :, None], shape).reshape(-1)
    for a in range(3):
        u[a][~mask] = 0.0
    rho = np.ones(N)
    zero = np.zeros(N)
    return _pack(rho, u, [zero, zero, zero, pxy, zero, zero])


# ---- round jet (Sec. 3.2 shape; grid 256 x 256 x 640, Re = 7000) ------------

def jet_params(nx=256, ny=256, nz=640, D=20, u_jet=0.05, re=7000.0, noise_amp=0.01, seed=3):
    """Inflow z = 0 (Hermite-NEE ghost), outflow z = nz-1, free-slip x and y walls.

    tau = 1/2 + nu / cs^2 with nu = u_jet D / Re; nozzle of diameter D centred
    at ((nx-1)/2, (ny-1)/2).
    """
    nu = u_jet * D / re
    tau = 0.5 + nu / CS2
    inflow = dict(center2=(nx - 1, ny - 1), diameter=D, u_jet=u_jet, noise_amp=noise_amp, seed=seed)
    return dict(dims=(nx, ny, nz), tau=tau, force=(0.0, 0.0, 0.0),
                bc=(FREESLIP, FREESLIP, FREESLIP, FREESLIP, INFLOW, OUTFLOW), inflow=inflow, nu=nu)


def jet_paper_params(nx=440, ny=440, nz=600, D=20, u_jet=0.05, re=7000.0, noise_amp=0.01, seed=3,
                     sponge_width=50, sponge_k=1000.0):
    """The paper's round-jet set-up (Sec. 3.2): 440 x 440 x 600, periodic crossflow
    (x and y), Hermite-NEE inflow at z = 0 with a uniform profile plus
    time-varying Gaussian noise, outflow at z = nz-1, and a sponge layer of
    width 50 and strength K = 1000 before the exit.  tau from Re = U D / nu.
    """
    nu = u_jet * D / re
    tau = 0.5 + nu / CS2
    inflow = dict(center2=(nx - 1, ny - 1), diameter=D, u_jet=u_jet, noise_amp=noise_amp, seed=seed,
                  noise="gaussian")
    return dict(dims=(nx, ny, nz), tau=tau, force=(0.0, 0.0, 0.0),
                bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC, INFLOW, OUTFLOW), inflow=inflow, nu=nu,
                sponge=(sponge_width, sponge_k))


# ---- D2Q9 channel (two-dimensional variant, 8192 x 2050) -----------------------

def channel2d_params(nx=8192, ny=2050, u_tau=0.0035, tau=0.503):
    """Bounce-back walls at y = 0 and y = ny-1 (solid layers), periodic x,
    H = (ny-2)/2, body force g = u_tau^2 / H along x.  16.78 M interior nodes at
    the default size (the same count as the three-dimensional channel)."""
    H = (ny - 2) / 2.0
    g = u_tau * u_tau / H
    return dict(dims=(nx, ny, 1), tau=tau, force=(g, 0.0, 0.0), bc=(PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK,
                                                                   PERIODIC, PERIODIC), H=H, u_tau=u_tau)


def channel2d_state(prm, seed=1, noise=0.02, re_tau=180.0):
    """Parabola to the log-law centreline speed plus uniform noise (as the 3-D
    channel), Pi from the parabola's shear; arrays in the three-dimensional
    layouts (u_z, Pi_zz, Pi_xz, Pi_yz zero)."""
    nx, ny, _ = prm["dims"]
    H, tau = prm["H"], prm["tau"]
    Uc = prm["u_tau"] * (math.log(re_tau) / 0.41 + 5.0)
    rng = np.random.default_rng(seed)
    N = nx * ny
    y = np.repeat(np.arange(ny, dtype=float), nx)
    eta = (y - 0.5) / (2.0 * H)  # walls halfway between the solid and first fluid layers
    ux = np.clip(4.0 * Uc * eta * (1.0 - eta), 0.0, None)
    u = np.zeros((3, N))
    u[0] = ux + noise * Uc * rng.uniform(-1.0, 1.0, N)
    u[1] = noise * Uc * rng.uniform(-1.0, 1.0, N)
    dudy = 4.0 * Uc * (1.0 - 2.0 * eta) / (2.0 * H)
    pi = np.zeros((6, N))
    pi[3] = -CS2 * tau * dudy
    return np.ones(N), u, pi


# ---- adjoint box (128^3 periodic, divergence-free random velocity) ----------

def divfree_random(n=128, u_rms=0.02, kmax=8, tau=0.52, seed=5):
    """Random solenoidal velocity from Fourier modes |k| <= kmax, projected, scaled to u_rms.

    Pi^neq from the spectral velocity gradient.  rho = 1.
    """
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    mask = (kk <= kmax) & (kk > 0)
    uh = [np.where(mask, rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape), 0.0) for _ in range(3)]
    ksafe = np.where(kk > 0, kk, 1.0)
    kv = (kx, ky, kz)
    div = (kx * uh[0] + ky * uh[1] + kz * uh[2]) / (ksafe ** 2)
    uh = [uh[a] - kv[a] * div for a in range(3)]
    u = [np.real(np.fft.ifftn(uh[a])) for a in range(3)]
    rms = math.sqrt(sum(float(np.mean(ua ** 2)) for ua in u) / 3.0)
    s = u_rms / rms
    u = [ua * s for ua in u]
    uh = [np.fft.fftn(ua) for ua in u]
    kw = [2.0 * math.pi / n * k for k in kv]
    grad = [[np.real(np.fft.ifftn(1j * kw[b] * uh[a])) for b in range(3)] for a in range(3)]  # d_b u_a
    c = -CS2 * tau
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    pi = [c * (grad[a][b] + grad[b][a]) for (a, b) in pairs]
    # arrays are indexed [z][y][x] already (meshgrid ij over z, y, x)
    rho = np.ones(n ** 3)
    return (n, n, n), _pack(rho, [ua.reshape(-1) for ua in u], [p.reshape(-1) for p in pi])
