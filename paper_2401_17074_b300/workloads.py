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


def _hash32(xp, k):
    """Integer hash of non-negative int64 values below 2^32 (two xorshift-multiply
    rounds with a multiplier below 2^31, so every product fits in int64); exact
    and identical for numpy arrays and torch tensors."""
    M = 0xFFFFFFFF
    k = ((k ^ (k >> 16)) * 0x45D9F3B) & M
    k = ((k ^ (k >> 16)) * 0x45D9F3B) & M
    return k ^ (k >> 16)


def hashed_moments(idx, seed, drho=2.0 ** -7, du=2.0 ** -5, dpi=2.0 ** -10):
    """Random moments at lattice node indices idx (int64 array, numpy or torch):
    rho - 1, u and Pi^neq from a counter hash of (idx, field, seed), uniform in
    [-amp, amp) with power-of-two amplitudes.  Every value is a multiple of
    2^-23 times its amplitude, so it is exact in FP32 and numpy and torch give
    identical bits.  Returns (drho [n], u [3, n], pi [6, n]) in FP32, for
    lattices too large to build on the host."""
    is_torch = type(idx).__module__.startswith("torch")
    out = []
    for f in range(10):
        key = (idx * 10 + f + 1000003 * seed) & 0xFFFFFFFF
        h = _hash32(None, key)
        q = (h >> 8) - (1 << 23)  # integer in [-2^23, 2^23)
        amp = drho if f == 0 else (du if f < 4 else dpi)
        scale = amp * 2.0 ** -23  # a power of two: q * scale is exact in FP32
        if is_torch:
            import torch
            out.append(q.to(torch.float32) * scale)
        else:
            out.append(q.astype(np.float32) * np.float32(scale))
    if is_torch:
        import torch
        return out[0], torch.stack(out[1:4]), torch.stack(out[4:])
    return out[0], np.stack(out[1:4]), np.stack(out[4:])


def channel_transition_state(prm, seed=2, streak=0.3, vortex=0.3, modes=0.1, noise=0.02):
    """A strongly disturbed channel flow meant to become turbulent quickly.

    Mean flow: Reichardt's smooth law of the wall for the Re_tau of the set-up
    (u+ = ln(1 + 0.4 y+)/0.4 + 7.8 (1 - exp(-y+/11) - (y+/11) exp(-y+/3)),
    y+ the distance to the nearer wall in wall units u_tau/nu).  On it, with
    s(y) = sin(pi eta), eta the fraction of the way across the channel, and
    U_c the centreline velocity:
      - streamwise streaks u' = streak U_c sin(beta z) s(y) cos(alpha x);
      - streamwise vortices from the stream function
        psi = vortex U_c s(y)^2 / beta cos(beta z), v = d psi/dz, w = -d psi/dy,
        both modulated along x by (1 + 0.5 cos(2 alpha x)) (still divergence-free
        in every x plane);
      - eight random large-scale modes per component, s(y) sin(k_x x + k_z z + phi)
        with k_x, k_z of 1 to 4 periods, of total amplitude `modes` U_c;
      - noise U_c xi, xi ~ U(-1, 1), on every component.
    beta gives a spanwise period near 100 wall units (a whole number of
    periods in z), alpha one period along x.  rho = 1 and Pi^neq from the mean
    shear.  Seeded."""
    nx, ny, nz = prm["dims"]
    H, tau, ut = prm["H"], prm["tau"], prm["u_tau"]
    nu = CS2 * (tau - 0.5)
    y0, y1 = 0.5, ny - 1.5
    yv = np.arange(ny, dtype=np.float64)
    dw = np.minimum(yv - y0, y1 - yv)  # distance to the nearer wall
    yp = np.maximum(dw, 0.0) * ut / nu
    up = np.log1p(0.4 * yp) / 0.4 + 7.8 * (1 - np.exp(-yp / 11) - (yp / 11) * np.exp(-yp / 3))
    U = ut * up
    Uc = float(U.max())
    dU = np.gradient(U, yv)
    fluid = (yv >= 1) & (yv <= ny - 2)
    U[~fluid] = 0.0
    dU[~fluid] = 0.0
    eta = np.clip((yv - y0) / (y1 - y0), 0.0, 1.0)
    s = np.sin(math.pi * eta)
    ds = math.pi / (y1 - y0) * np.cos(math.pi * eta)
    nper = max(1, round(nz * ut / (100.0 * nu)))  # spanwise periods of about 100 wall units
    beta = 2 * math.pi * nper / nz
    alpha = 2 * math.pi / nx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    S, dS = s[y], ds[y]
    fx = 1.0 + 0.5 * np.cos(2 * alpha * x)
    ux = U[y] + streak * Uc * np.sin(beta * z) * S * np.cos(alpha * x)
    uy = -vortex * Uc * np.sin(beta * z) * S * S * fx
    uz = -vortex * Uc / beta * np.cos(beta * z) * 2 * S * dS * fx
    rng = np.random.default_rng(seed)
    u = [ux, uy, uz]
    for a in range(3):
        for _ in range(8):
            kx = 2 * math.pi * rng.integers(1, 5) / nx
            kz = 2 * math.pi * rng.integers(1, 5) / nz
            u[a] = u[a] + (modes / 8.0) * Uc * S * np.sin(kx * x + kz * z + rng.uniform(0, 2 * math.pi))
    u = [c.reshape(-1) for c in u]
    mask = np.broadcast_to(fluid[None, :, None], (nz, ny, nx)).reshape(-1)
    for a in range(3):
        u[a] = u[a] + noise * Uc * rng.uniform(-1.0, 1.0, u[a].size)
        u[a][~mask] = 0.0
    N = nx * ny * nz
    pxy = np.broadcast_to((-CS2 * tau * dU)[None, :, None], (nz, ny, nx)).reshape(-1).copy()
    zero = np.zeros(N)
    return np.ones(N), np.stack(u), np.stack([zero, zero, zero, pxy, zero, zero])
