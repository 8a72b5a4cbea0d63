"""Parity at the full workload sizes, in the launch configuration bench.py times.

The CUDA step runs on the whole lattice (turbulent channel 512 x 130 x 256,
round jet 256 x 256 x 640) with the default kernel and FP32 storage.  The
oracle cannot run those lattices, so it recomputes sampled columns one by one:
after k steps a node depends only on nodes within distance k, so a small
oracle box cut out around the column (periodic axes wrapped, wall layers kept,
one extra fake wall layer beyond the dependency radius where the box is cut
inside the fluid) reproduces that column exactly.  Samples sit on tile
boundaries, periodic seams, walls and the nozzle.
"""
import numpy as np
import pytest

import oracle
import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

NSTEPS = 2


def _cut(arr, dims, xs, ys, zs):
    """Full-lattice [..., N] array (numpy, or a CUDA tensor) -> numpy sub-box [..., n] over index lists xs, ys, zs."""
    nx, ny, nz = dims
    if hasattr(arr, "is_cuda"):
        import torch
        dev = arr.device
        a = arr.reshape(tuple(arr.shape[:-1]) + (nz, ny, nx))
        a = a.index_select(-3, torch.as_tensor(zs, device=dev)).index_select(-2, torch.as_tensor(ys, device=dev))
        a = a.index_select(-1, torch.as_tensor(xs, device=dev))
        return a.reshape(tuple(arr.shape[:-1]) + (-1,)).cpu().numpy()
    a = arr.reshape(arr.shape[:-1] + (nz, ny, nx))
    a = a[..., zs, :, :][..., :, ys, :][..., :, :, xs]
    return np.ascontiguousarray(a.reshape(arr.shape[:-1] + (-1,)))


def _axis_range(c, n, periodic, R):
    """Lattice indices of a sub-box axis around c, and whether it is periodic."""
    if periodic:
        return [(c + d) % n for d in range(-R, R + 1)], True
    lo, hi = max(0, c - R - 1), min(n - 1, c + R + 1)
    return list(range(lo, hi + 1)), False


def _compare_column(gpu, state_full, dims, tau, force, bc, col, inflow=None, sponge=None):
    """Run the oracle on the sub-box around column `col` and compare that column.

    col: dict with the two sampled coordinates (the third axis is kept whole).
    """
    nx, ny, nz = dims
    R = NSTEPS
    axes = []
    for a, n in enumerate(dims):
        per = bc[2 * a] == 0
        if a in col:
            idx, p = _axis_range(col[a], n, per, R)
        else:
            idx, p = list(range(n)), per
        axes.append((idx, p))
    xs, ys, zs = axes[0][0], axes[1][0], axes[2][0]
    sdims = (len(xs), len(ys), len(zs))
    sbc = []
    for a in range(3):
        if axes[a][1]:
            sbc += [0, 0]
        else:
            sbc += [bc[2 * a], bc[2 * a + 1]]
    rho, u, pi = state_full
    sub = (_cut(rho, dims, xs, ys, zs), _cut(u, dims, xs, ys, zs), _cut(pi, dims, xs, ys, zs))
    sin = None
    if inflow is not None:
        sin = dict(inflow)
        sin["origin"] = (xs[0], ys[0])
    o = oracle.OracleSim(sdims, tau, force=force, bc=tuple(sbc), inflow=sin, sponge=sponge)
    o.init_moments(*sub)
    o.step(NSTEPS)
    r, uu, pp = o.get_moments()
    ref = np.concatenate([(r - 1)[None], uu, pp])
    got = _cut(gpu, dims, xs, ys, zs)
    # positions of the sampled column inside the sub-box
    sel = np.zeros((sdims[2], sdims[1], sdims[0]), bool)
    ix = xs.index(col[0]) if 0 in col else slice(None)
    iy = ys.index(col[1]) if 1 in col else slice(None)
    iz = zs.index(col[2]) if 2 in col else slice(None)
    sel[iz, iy, ix] = True
    # interior of the full lattice only (per axis: not a boundary layer)
    keep = []
    for a, idx in enumerate((xs, ys, zs)):
        n = dims[a]
        keep.append(np.array([bc[2 * a] == 0 or 0 < i < n - 1 for i in idx]))
    inner_sub = keep[2][:, None, None] & keep[1][None, :, None] & keep[0][None, None, :]
    m = sel.reshape(-1) & inner_sub.reshape(-1)
    return got[:, m], ref[:, m]


def _run_gpu(prm, state, inflow=None):
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], inflow=inflow)
    s.init_moments(*state)
    s.step(NSTEPS)
    r, u, p = s.get_moments()
    s.close()
    return np.concatenate([(r - 1)[None], u, p])


def _check(pairs, tol, tol_drho=2e-5, tol_pi=None):
    """Relative L2 errors over the sampled nodes, per field group.

    u and Pi^neq are compared as tensors (error norm over all components
    against the norm of the whole tensor): single components can start at
    exactly zero (the channel's Pi_xx, Pi_yy, Pi_zz) and are then meaningless
    as relative errors.  rho - 1 is a small difference of cancelling mass
    fluxes (the channel starts at rho = 1 exactly), so its FP32 floor relative
    to its own norm is higher; it gets the same 2e-5 bound as in the
    Taylor-Green parity test.
    """
    got = np.concatenate([g for g, _ in pairs], axis=1)
    ref = np.concatenate([r for _, r in pairs], axis=1)
    tol_pi = tol if tol_pi is None else tol_pi
    for name, rows, bound in (("drho", [0], tol_drho), ("u", [1, 2, 3], tol), ("pi", [4, 5, 6, 7, 8, 9], tol_pi)):
        err = np.linalg.norm(got[rows] - ref[rows]) / np.linalg.norm(ref[rows])
        assert err <= bound, (name, err)


def _oracle_full(prm, state, inflow=None):
    o = oracle.OracleSim(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], inflow=inflow)
    o.init_moments(*state)
    o.step(NSTEPS)
    r, u, p = o.get_moments()
    return np.concatenate([(r - 1)[None], u, p])


def test_subbox_columns_reproduce_full_oracle():
    """The column sampler itself: sub-box recomputation equals a full oracle run (CPU)."""
    prm = W.channel_params(nx=14, ny=12, nz=9)
    state = W.channel_state(prm, seed=3)
    full = _oracle_full(prm, state)
    for col in ({0: 0, 2: 0}, {0: 13, 2: 4}, {0: 6, 2: 8}):
        got, ref = _compare_column(full, state, prm["dims"], prm["tau"], prm["force"], prm["bc"], col)
        assert np.abs(got - ref).max() < 1e-15
    prm = W.jet_params(nx=14, ny=13, nz=10, D=6)
    state = W.random_state(prm["dims"], seed=4, drho=0.002, du=0.01, dpi=1e-4)
    full = _oracle_full(prm, state, inflow=prm["inflow"])
    for col in ({0: 1, 1: 1}, {0: 12, 1: 6}, {0: 7, 1: 6}, {0: 4, 1: 11}):
        got, ref = _compare_column(full, state, prm["dims"], prm["tau"], prm["force"], prm["bc"], col,
                                   inflow=prm["inflow"])
        assert np.abs(got - ref).max() < 1e-15


@pytest.mark.gpu
def test_channel_full_size_sampled(cuda_ok):
    prm = W.channel_params()  # 512 x 130 x 256
    state = W.channel_state(prm, seed=1)
    gpu = _run_gpu(prm, state)
    cols = [{0: 0, 2: 0}, {0: 511, 2: 255}, {0: 255, 2: 128}, {0: 30, 2: 17}, {0: 29, 2: 200}, {0: 480, 2: 64}]
    pairs = [_compare_column(gpu, state, prm["dims"], prm["tau"], prm["force"], prm["bc"], c) for c in cols]
    # Pi^neq = sum f c c - rho u u - ... is here ~36x smaller than the rho u u
    # terms it is computed from (u_x ~ 0.06, Pi ~ 1e-4), so its FP32 floor after
    # two steps is ~1e-5 relative; u keeps the 3e-6 bound.
    _check(pairs, 3e-6, tol_pi=2e-5)


@pytest.mark.gpu
def test_channel_nee_walls_full_size_sampled(cuda_ok):
    """The bench channel with thread-safe NEE no-slip walls instead of bounce-back."""
    prm = dict(W.channel_params())  # 512 x 130 x 256
    prm["bc"] = (0, 0, 5, 5, 0, 0)
    state = W.channel_state(prm, seed=1)
    gpu = _run_gpu(prm, state)
    cols = [{0: 0, 2: 0}, {0: 511, 2: 255}, {0: 255, 2: 128}, {0: 30, 2: 17}, {0: 29, 2: 200}]
    pairs = [_compare_column(gpu, state, prm["dims"], prm["tau"], prm["force"], prm["bc"], c) for c in cols]
    _check(pairs, 3e-6, tol_pi=2e-5)


@pytest.mark.gpu
def test_jet_full_size_sampled(cuda_ok):
    prm = W.jet_params()  # 256 x 256 x 640, inflow z = 0, outflow z = 639, free-slip sides
    dims = prm["dims"]
    # small random deviations from rest exercise every term of the step
    state = W.random_state(dims, seed=41, drho=0.002, du=0.01, dpi=1e-4)
    gpu = _run_gpu(prm, state, inflow=prm["inflow"])
    cols = [{0: 1, 1: 1}, {0: 1, 1: 128}, {0: 254, 1: 254}, {0: 127, 1: 128}, {0: 118, 1: 127}, {0: 200, 1: 50},
            {0: 30, 1: 17}]
    pairs = [_compare_column(gpu, state, dims, prm["tau"], prm["force"], prm["bc"], c, inflow=prm["inflow"])
             for c in cols]
    _check(pairs, 3e-6)


@pytest.mark.gpu
def test_paper_jet_full_size_sampled(cuda_ok):
    """The paper's jet at its own size (Sec. 3.2: 440 x 440 x 600, periodic
    crossflow, Gaussian inflow noise, sponge of width 50 with K = 1000).  The
    state is drawn on the device from a seeded generator, so no full-lattice
    host copy is made; sampled columns span every z, through the sponge."""
    import torch
    prm = W.jet_paper_params()
    dims = prm["dims"]
    N = dims[0] * dims[1] * dims[2]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(51)

    def unif(shape, scale):
        return (torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64) * 2.0 - 1.0) * scale

    rho = 1.0 + unif((N,), 0.002)
    u = unif((3, N), 0.01)
    pi = unif((6, N), 1e-4)
    s = T.Solver(dims, prm["tau"], force=prm["force"], bc=prm["bc"], inflow=prm["inflow"], sponge=prm["sponge"])
    s.init_moments(rho, u, pi)
    s.step(NSTEPS)
    out = torch.empty((10, N), dtype=torch.float64, device="cuda")
    T.tslb_get_moments(s.handle, out[0], out[1:4], out[4:10], T.DEVICE)
    s.close()
    out[0] -= 1.0
    cols = [{0: 219, 1: 219}, {0: 210, 1: 223}, {0: 0, 1: 0}, {0: 439, 1: 100}, {0: 30, 1: 17}, {0: 300, 1: 431}]
    pairs = [_compare_column(out, (rho, u, pi), dims, prm["tau"], prm["force"], prm["bc"], c, inflow=prm["inflow"],
                             sponge=prm["sponge"]) for c in cols]
    _check(pairs, 3e-6)


@pytest.mark.gpu
def test_bf16_lattice_beyond_2_31_nodes(cuda_ok):
    """A BF16 lattice of 1024 x 1024 x 2049 = 2,148,532,224 nodes (more than
    2^31; 86 GB for the two moment buffers) runs the factored kernel, and three
    sampled z columns after two steps match the oracle on their cut-out boxes:
    (0, 0), whose layer z = 2048 starts at node 2^31, (1023, 1023), which
    ends at node 2^31 - 1 in layer 2047, and one inside.  The input is the
    counter-hashed random state (exact in FP32 on both sides), built on the
    device in chunks.  Bounds as for 16-bit storage elsewhere: u 4 units of
    BF16 roundoff, Pi 16 (relative L2 over the column)."""
    import torch
    dims = (1024, 1024, 2049)
    nx, ny, nz = dims
    N = nx * ny * nz
    assert N > 2 ** 31
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.skip("needs about 180 GB of free device memory")
    tau, seed = 0.6, 7
    s = T.Solver(dims, tau, precision=T.BF16, u_ref=0.05, pi_ref=2.0 ** -9, kernel=T.KERNEL_FACTORED)
    dev = "cuda"
    drho = torch.empty(N, dtype=torch.float32, device=dev)
    u = torch.empty((3, N), dtype=torch.float32, device=dev)
    pi = torch.empty((6, N), dtype=torch.float32, device=dev)
    chunk = nx * ny * 64
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        r0, u0, p0 = W.hashed_moments(torch.arange(a, b, dtype=torch.int64, device=dev), seed)
        drho[a:b] = r0
        u[:, a:b] = u0
        pi[:, a:b] = p0
    T.tslb_init_moments_f32(s.handle, drho, u, pi)
    s.step(NSTEPS)
    T.tslb_get_moments_f32(s.handle, drho, u, pi, T.DEVICE)
    torch.cuda.synchronize()
    s.close()
    R = NSTEPS
    ur = 2.0 ** -8  # BF16 unit roundoff
    for cx, cy in ((0, 0), (nx - 1, ny - 1), (511, 700)):
        xs = [(cx + d) % nx for d in range(-R, R + 1)]
        ys = [(cy + d) % ny for d in range(-R, R + 1)]
        zz, yy, xx = np.meshgrid(np.arange(nz), ys, xs, indexing="ij")
        gidx = (xx + nx * (yy + ny * zz)).reshape(-1).astype(np.int64)
        r0, u0, p0 = W.hashed_moments(gidx, seed)
        o = oracle.OracleSim((len(xs), len(ys), nz), tau)
        o.init_moments(1.0 + r0.astype(np.float64), u0.astype(np.float64), p0.astype(np.float64))
        o.step(NSTEPS)
        r, uu, pp = o.get_moments()
        ref = np.concatenate([(r - 1)[None], uu, pp]).reshape(10, nz, len(ys), len(xs))[:, :, R, R]
        col = torch.as_tensor(cx + nx * (cy + ny * np.arange(nz, dtype=np.int64)), device=dev)
        got = torch.cat([drho[col][None], u[:, col], pi[:, col]]).double().cpu().numpy()
        eu = np.linalg.norm(got[1:4] - ref[1:4]) / np.linalg.norm(ref[1:4])
        ep = np.linalg.norm(got[4:] - ref[4:]) / np.linalg.norm(ref[4:])
        er = np.linalg.norm(got[0] - ref[0]) / np.linalg.norm(ref[0])
        print("column (%d, %d): drho %.2e u %.2e Pi %.2e" % (cx, cy, er, eu, ep))
        assert eu <= 4 * ur and er <= 4 * ur and ep <= 16 * ur, (cx, cy, er, eu, ep)
