"""Discrete adjoint of the TSLB step against the oracle's complex-step gradient.

J = 1/2 sum rho |u|^2 after 64 steps on a periodic box (and on small channel
boxes with bounce-back y walls) from a seeded
divergence-free random velocity (tau = 0.52); control = per-node body-force
field F (zero).  Directional derivatives <dJ/dF, v> from the GPU adjoint
(checkpoint every 16 steps, FP32) must agree with Im J(F + i h v) / h of the
FP64 oracle (h = 1e-30) to 1e-4 relative.
"""
import numpy as np
import pytest

import oracle
import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(n, nsteps=64, k=16, tau=0.52):
    dims, state = W.divfree_random(n=n, u_rms=0.02, kmax=min(8, n // 3), tau=tau, seed=5)
    s = T.Solver(dims, tau, checkpoint_every=k)
    return dims, state, s


@pytest.mark.parametrize("n", [8, 16])
def test_adjoint_matches_complex_step(cuda_ok, n):
    nsteps, tau = 64, 0.52
    dims, state, s = _setup(n, nsteps=nsteps, tau=tau)
    N = n ** 3
    F0 = np.zeros((3, N), dtype=np.float32)
    s.init_moments(*state)
    s.set_force_field(F0)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64)
    s.close()
    rng = np.random.default_rng(17)
    for trial in range(3):
        v = rng.standard_normal((3, N))
        h = 1e-30
        J = oracle.complex_step_energy(dims, tau, (0,) * 6, state[0], state[1], state[2], F0.astype(np.float64),
                                       h * v, nsteps)
        d_cs = J.imag / h
        d_adj = float(np.sum(g * v))
        assert abs(d_adj - d_cs) <= 1e-4 * abs(d_cs), (trial, d_adj, d_cs)


def _complex_step_entry(dims, tau, state, F0, nsteps, a, i):
    """dJ/dF_a(node i) of the FP64 oracle by the complex step."""
    v = np.zeros((3, dims[0] * dims[1] * dims[2]))
    v[a, i] = 1.0
    h = 1e-30
    J = oracle.complex_step_energy(dims, tau, (0,) * 6, state[0], state[1], state[2], F0.astype(np.float64), h * v,
                                   nsteps)
    return J.imag / h


def test_adjoint_every_entry_small_box(cuda_ok):
    """Every entry of the 3 x 4^3 gradient against the oracle's complex step
    (a random force field, 16 steps, checkpoints every 4): entry by entry, so
    an error confined to a few nodes or one component cannot hide in a
    random projection."""
    n, nsteps, tau = 4, 16, 0.55
    dims, state = W.divfree_random(n=n, u_rms=0.02, kmax=1, tau=tau, seed=5)
    N = n ** 3
    F0 = (1e-5 * np.random.default_rng(41).uniform(-1, 1, (3, N))).astype(np.float32)
    s = T.Solver(dims, tau, checkpoint_every=4)
    s.set_force_field(F0)
    s.init_moments(*state)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64).reshape(3, N)
    s.close()
    cs = np.array([[_complex_step_entry(dims, tau, state, F0, nsteps, a, i) for i in range(N)] for a in range(3)])
    assert np.abs(g - cs).max() <= 1e-4 * np.abs(cs).max(), np.abs(g - cs).max() / np.abs(cs).max()
    assert np.linalg.norm(g - cs) <= 1e-4 * np.linalg.norm(cs)


def test_adjoint_single_entries_16(cuda_ok):
    """Twelve single entries (random component and node) of the 3 x 16^3
    gradient of the 64-step workload against the oracle's complex step, each
    within 1e-4 of its own size (floor: 1 % of the largest entry)."""
    n, nsteps, tau = 16, 64, 0.52
    dims, state, s = _setup(n, nsteps=nsteps, tau=tau)
    N = n ** 3
    F0 = np.zeros((3, N), dtype=np.float32)
    s.init_moments(*state)
    s.set_force_field(F0)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64).reshape(3, N)
    s.close()
    rng = np.random.default_rng(43)
    gmax = np.abs(g).max()
    for a, i in zip(rng.integers(0, 3, 12), rng.integers(0, N, 12)):
        cs = _complex_step_entry(dims, tau, state, F0, nsteps, int(a), int(i))
        assert abs(g[a, i] - cs) <= 1e-4 * max(abs(cs), 0.01 * gmax), (a, i, g[a, i], cs)


def _oracle_energy(dims, tau, state, F, nsteps):
    o = oracle.OracleSim(dims, tau)
    o.init_moments(*state)
    o.set_force_field(F)
    o.step(nsteps)
    r, u, _ = o.get_moments()
    return 0.5 * float(np.sum(r * (u ** 2).sum(0)))


def test_adjoint_matches_central_differences(cuda_ok):
    """16^3, 64 steps: the GPU adjoint's directional derivative against FP64
    central differences of the oracle, (J(F + eps v) - J(F - eps v)) / (2 eps)
    with eps = 1e-6 (truncation O(eps^2), far below the bound)."""
    n, nsteps, tau = 16, 64, 0.52
    dims, state, s = _setup(n, nsteps=nsteps, tau=tau)
    N = n ** 3
    F0 = np.zeros((3, N), dtype=np.float32)
    s.init_moments(*state)
    s.set_force_field(F0)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64)
    s.close()
    v = np.random.default_rng(18).standard_normal((3, N))
    eps = 1e-6
    d_fd = (_oracle_energy(dims, tau, state, eps * v, nsteps) - _oracle_energy(dims, tau, state, -eps * v, nsteps)) / (
        2 * eps)
    d_adj = float(np.sum(g * v))
    assert abs(d_adj - d_fd) <= 1e-4 * abs(d_fd), (d_adj, d_fd)


def test_adjoint_matches_complex_step_128(cuda_ok):
    """The full-size adjoint workload: 128^3, 64 steps, checkpoints every 16,
    one random direction against the oracle's complex-step derivative (about a
    minute of host time for the complex-step run)."""
    n, nsteps, tau = 128, 64, 0.52
    dims, state, s = _setup(n, nsteps=nsteps, tau=tau)
    N = n ** 3
    F0 = np.zeros((3, N), dtype=np.float32)
    s.init_moments(*state)
    s.set_force_field(F0)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64)
    s.close()
    v = np.random.default_rng(17).standard_normal((3, N))
    h = 1e-30
    J = oracle.complex_step_energy(dims, tau, (0,) * 6, state[0], state[1], state[2], F0.astype(np.float64), h * v,
                                   nsteps)
    d_cs = J.imag / h
    d_adj = float(np.sum(g * v))
    assert abs(d_adj - d_cs) <= 1e-4 * abs(d_cs), (d_adj, d_cs)


@pytest.mark.parametrize("dims", [(70, 9, 5), (68, 7, 5)], ids=["cell-copies", "row-copies"])
def test_adjoint_ragged_box_with_force(cuda_ok, dims):
    """Boxes that the gather's 32 x 4 x 2 blocks do not tile (ragged blocks on
    every axis, x wider than a block, so the halo wraps in one step), a nonzero
    random force field, and checkpoint segments of 8, 8 and 4 steps.  70 x 9 x 5
    takes the per-cell tile load; 68 x 7 x 5 (nx a multiple of 4) the 16-byte
    row copies, whose last block's columns wrap to x = 0."""
    tau, nsteps = 0.55, 20
    N = dims[0] * dims[1] * dims[2]
    state = W.random_state(dims, seed=38, drho=0.002, du=0.02, dpi=1e-4)
    F0 = (1e-5 * np.random.default_rng(39).uniform(-1, 1, (3, N))).astype(np.float32)
    s = T.Solver(dims, tau, checkpoint_every=8)
    s.set_force_field(F0)
    s.init_moments(*state)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64)
    s.close()
    rng = np.random.default_rng(40)
    for trial in range(2):
        v = rng.standard_normal((3, N))
        h = 1e-30
        J = oracle.complex_step_energy(dims, tau, (0,) * 6, state[0], state[1], state[2], F0.astype(np.float64),
                                       h * v, nsteps)
        d_cs = J.imag / h
        d_adj = float(np.sum(g * v))
        assert abs(d_adj - d_cs) <= 1e-4 * abs(d_cs), (trial, d_adj, d_cs)


@pytest.mark.parametrize("dims", [(40, 10, 6), (13, 9, 5)], ids=["row-copies", "cell-copies"])
def test_adjoint_bounce_back_walls(cuda_ok, dims):
    """The channel's halfway bounce-back y walls (8 and 7 interior rows, so
    ragged against the 4-row gather blocks), a random force field and
    checkpoint segments of 4 steps: directional derivatives against the
    oracle's complex step, and zero gradient on the wall layers."""
    tau, nsteps, bc = 0.6, 12, (0, 0, 1, 1, 0, 0)
    N = dims[0] * dims[1] * dims[2]
    state = W.random_state(dims, seed=44, drho=0.002, du=0.02, dpi=1e-4)
    F0 = (1e-5 * np.random.default_rng(45).uniform(-1, 1, (3, N))).astype(np.float32)
    s = T.Solver(dims, tau, bc=bc, checkpoint_every=4)
    s.set_force_field(F0)
    s.init_moments(*state)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64)
    s.close()
    walls = g.reshape(3, dims[2], dims[1], dims[0])[:, :, [0, -1], :]
    assert np.all(walls == 0)
    rng = np.random.default_rng(46)
    for trial in range(2):
        v = rng.standard_normal((3, N))
        h = 1e-30
        J = oracle.complex_step_energy(dims, tau, bc, state[0], state[1], state[2], F0.astype(np.float64), h * v,
                                       nsteps)
        d_cs = J.imag / h
        d_adj = float(np.sum(g * v))
        assert abs(d_adj - d_cs) <= 1e-4 * abs(d_cs), (trial, d_adj, d_cs)


def test_adjoint_bounce_back_every_entry(cuda_ok):
    """Every interior entry of the gradient on a 4 x (4 + 2) x 4 channel box
    with bounce-back y walls against the oracle's complex step."""
    dims, tau, nsteps, bc = (4, 6, 4), 0.6, 16, (0, 0, 1, 1, 0, 0)
    N = dims[0] * dims[1] * dims[2]
    state = W.random_state(dims, seed=47, drho=0.002, du=0.02, dpi=1e-4)
    F0 = (1e-5 * np.random.default_rng(48).uniform(-1, 1, (3, N))).astype(np.float32)
    s = T.Solver(dims, tau, bc=bc, checkpoint_every=4)
    s.set_force_field(F0)
    s.init_moments(*state)
    s.step(nsteps)
    g = s.adjoint_force_gradient(nsteps).astype(np.float64).reshape(3, N)
    s.close()
    y = (np.arange(N) // dims[0]) % dims[1]
    interior = np.nonzero((y > 0) & (y < dims[1] - 1))[0]
    cs = np.zeros((3, N))
    for a in range(3):
        for i in interior:
            v = np.zeros((3, N))
            v[a, i] = 1.0
            J = oracle.complex_step_energy(dims, tau, bc, state[0], state[1], state[2], F0.astype(np.float64),
                                           1e-30 * v, nsteps)
            cs[a, i] = J.imag / 1e-30
    assert np.abs(g - cs).max() <= 1e-4 * np.abs(cs).max(), np.abs(g - cs).max() / np.abs(cs).max()


@pytest.mark.parametrize("prec, ur", [(T.BF16, 2.0 ** -8), (T.FP16, 2.0 ** -11)], ids=["bf16", "fp16"])
def test_adjoint_16bit_storage(cuda_ok, prec, ur):
    """With 16-bit moment storage the adjoint differentiates the FP32 step
    arithmetic along the stored (rounded) trajectory.  Each step rounds every
    stored value once (unit roundoff ur); the gradient is a smooth function of
    that trajectory, and its relative L2 difference from the FP32 run's is of
    the order of one rounding (measured 0.67 ur for BF16 and for FP16 at 16^3,
    64 steps: the roundings do not accumulate like a random walk).  Bound:
    4 ur."""
    n, nsteps, tau = 16, 64, 0.52
    grads = {}
    for p in (T.FP32, prec):
        dims, state = W.divfree_random(n=n, u_rms=0.02, kmax=5, tau=tau, seed=5)
        s = T.Solver(dims, tau, checkpoint_every=16, precision=p, u_ref=0.05, pi_ref=W.pi_reference(state))
        s.init_moments(*state)
        s.set_force_field(np.zeros((3, n ** 3), dtype=np.float32))
        s.step(nsteps)
        grads[p] = s.adjoint_force_gradient(nsteps).astype(np.float64)
        s.close()
    err = np.linalg.norm(grads[prec] - grads[T.FP32]) / np.linalg.norm(grads[T.FP32])
    assert err <= 4 * ur, err


def test_adjoint_rejects_other_faces(cuda_ok):
    s = T.Solver((8, 8, 8), 0.6, bc=(2, 2, 0, 0, 0, 0), checkpoint_every=4)  # free-slip x faces
    s.init_moments(*W.random_state((8, 8, 8), seed=49))
    s.step(4)
    with pytest.raises(T.TslbError) as ei:
        s.adjoint_force_gradient(4)
    assert ei.value.code == T.TSLB_ERR_UNSUPPORTED
    s.close()


def test_adjoint_partial_window_and_errors(cuda_ok):
    n = 8
    dims, state, s = _setup(n)
    s.init_moments(*state)
    s.set_force_field(np.zeros((3, n ** 3), dtype=np.float32))
    s.step(40)
    with pytest.raises(T.TslbError) as ei:
        s.adjoint_force_gradient(30)  # 40 - 30 is not a multiple of 16
    assert ei.value.code == T.TSLB_ERR_INVALID
    g = s.adjoint_force_gradient(24)  # window [16, 40)
    assert np.all(np.isfinite(g)) and np.abs(g).max() > 0
    s.close()
    s2 = T.Solver(dims, 0.52)  # no checkpoints
    s2.init_moments(*state)
    s2.step(4)
    with pytest.raises(T.TslbError) as ei:
        s2.adjoint_force_gradient(4)
    assert ei.value.code == T.TSLB_ERR_STATE
    s2.close()


def test_autograd_function(cuda_ok):
    import torch
    from paper_2401_17074_b300.autograd import kinetic_energy
    n, nsteps = 8, 32
    dims, state, s = _setup(n, nsteps=nsteps)
    F = torch.zeros((3, n ** 3), dtype=torch.float32, device="cuda", requires_grad=True)
    J = kinetic_energy(F, s, state, nsteps)
    J.backward()
    g_auto = F.grad.detach().cpu().numpy()
    g_abi = s.adjoint_force_gradient(nsteps)
    assert np.array_equal(g_auto, g_abi)
    rho, u, _ = s.get_moments()
    assert abs(J.item() - 0.5 * np.sum(rho * (u ** 2).sum(0))) < 1e-9
    s.close()


def _profile_weights(dims, seed):
    """Random weights w_y of the plane-averaged u_x(y) profile over the interior rows."""
    w = np.random.default_rng(seed).standard_normal(dims[1])
    return w


def _objective_np(dims, bc, w, W10, rho, u, pi):
    """J(m) on (possibly complex) full-lattice moments, numpy: the u_x(y)
    profile averaged over x and z and weighted by w, plus sum W10 . m over all
    ten fields, plus 1/2 sum rho u_y^2.  Holomorphic (no conjugates), so the
    complex step differentiates it."""
    nx, ny, nz = dims
    ux = u[0].reshape(nz, ny, nx)
    prof = ux.mean(axis=(0, 2))
    y0, y1 = (1, ny - 1) if bc[2] != 0 else (0, ny)
    J = np.sum(w[y0:y1] * prof[y0:y1])
    m = np.concatenate([rho.reshape(1, -1), u, pi], axis=0)
    J = J + np.sum(W10 * m) + 0.5 * np.sum(rho * u[1] ** 2)
    return J


def _objective_torch(dims, bc, w, W10, rho, u, pi):
    import torch
    nx, ny, nz = dims
    prof = u[0].view(nz, ny, nx).mean(dim=(0, 2))
    y0, y1 = (1, ny - 1) if bc[2] != 0 else (0, ny)
    wt = torch.as_tensor(w, dtype=torch.float64, device=u.device)
    J = torch.sum(wt[y0:y1] * prof[y0:y1])
    m = torch.cat([rho.view(1, -1), u, pi], dim=0)
    J = J + torch.sum(torch.as_tensor(W10, device=u.device) * m) + 0.5 * torch.sum(rho * u[1] ** 2)
    return J


@pytest.mark.parametrize("case", ["periodic16", "channel"])
def test_adjoint_general_objective(cuda_ok, case):
    """A second objective through tslb_adjoint and the autograd Function that
    returns the final moments: the plane-averaged u_x(y) profile weighted by a
    random vector, plus a random linear functional of all ten moment fields,
    plus 1/2 sum rho u_y^2.  torch builds the cotangent of the final moments;
    the library's adjoint maps it to dJ/dF.  Directional derivatives must
    agree with the oracle's complex step of the same objective to 1e-4
    relative, on a 16^3 periodic box (64 steps, checkpoints every 16) and on a
    40 x 10 x 6 channel box with bounce-back y walls (12 steps, every 4)."""
    import torch
    from paper_2401_17074_b300.autograd import final_moments
    if case == "periodic16":
        n, nsteps, tau, k, bc = 16, 64, 0.52, 16, (0,) * 6
        dims, state = W.divfree_random(n=n, u_rms=0.02, kmax=5, tau=tau, seed=5)
    else:
        dims, tau, nsteps, k, bc = (40, 10, 6), 0.6, 12, 4, (0, 0, 1, 1, 0, 0)
        state = W.random_state(dims, seed=44, drho=0.002, du=0.02, dpi=1e-4)
    N = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(91)
    w = _profile_weights(dims, 92)
    W10 = 1e-3 * rng.standard_normal((10, N))
    F0 = (1e-5 * rng.uniform(-1, 1, (3, N))).astype(np.float32)
    s = T.Solver(dims, tau, bc=bc, checkpoint_every=k)
    F = torch.tensor(F0, device="cuda", requires_grad=True)
    rho, u, pi = final_moments(F, s, state, nsteps)
    J = _objective_torch(dims, bc, w, W10, rho, u, pi)
    J.backward()
    g = F.grad.detach().cpu().numpy().astype(np.float64)
    s.close()
    # the forward value against the oracle's real run of the same objective
    r0, u0, p0 = oracle.complex_step_moments(dims, tau, bc, state[0], state[1], state[2], F0.astype(np.float64),
                                             np.zeros((3, N)), nsteps)
    J_or = _objective_np(dims, bc, w, W10, r0, u0, p0).real
    assert abs(J.item() - J_or) <= 1e-5 * (abs(J_or) + 1e-3)
    for trial in range(2):
        v = rng.standard_normal((3, N))
        h = 1e-30
        rc, uc, pc = oracle.complex_step_moments(dims, tau, bc, state[0], state[1], state[2], F0.astype(np.float64),
                                                 h * v, nsteps)
        d_cs = _objective_np(dims, bc, w, W10, rc, uc, pc).imag / h
        d_adj = float(np.sum(g * v))
        assert abs(d_adj - d_cs) <= 1e-4 * abs(d_cs), (trial, d_adj, d_cs)


def test_adjoint_cotangent_reproduces_kinetic_energy_seed(cuda_ok):
    """tslb_adjoint with the cotangent of J = 1/2 sum rho |u|^2, that is
    (|u|^2 / 2, rho u, 0) built on the host from the final moments, gives the
    gradient of tslb_adjoint_force_gradient (the seed on the device) up to the
    FP32 rounding of the seed: 1e-6 relative in L2.  Also from device arrays."""
    import torch
    n, nsteps = 8, 32
    dims, state, s = _setup(n, nsteps=nsteps)
    N = n ** 3
    s.init_moments(*state)
    s.set_force_field(np.zeros((3, N), dtype=np.float32))
    s.step(nsteps)
    g_ke = s.adjoint_force_gradient(nsteps).astype(np.float64)
    rho, u, pi = s.get_moments()
    lam = np.concatenate([0.5 * (u ** 2).sum(0), (rho * u).reshape(-1), np.zeros(6 * N)])
    g_host = s.adjoint(lam, nsteps).astype(np.float64)
    lam_d = torch.tensor(lam, device="cuda")
    g_dev = torch.empty((3, N), dtype=torch.float32, device="cuda")
    T.tslb_adjoint(s.handle, lam_d, nsteps, 16, g_dev, T.DEVICE)
    s.close()
    assert np.linalg.norm(g_host - g_ke) <= 1e-6 * np.linalg.norm(g_ke)
    assert np.array_equal(g_dev.cpu().numpy(), g_host.astype(np.float32))


def test_adjoint_cotangent_errors(cuda_ok):
    n = 8
    dims, state, s = _setup(n)
    N = n ** 3
    s.init_moments(*state)
    s.set_force_field(np.zeros((3, N), dtype=np.float32))
    s.step(16)
    lam = np.zeros(10 * N)
    g = np.zeros(3 * N, dtype=np.float32)
    with pytest.raises(T.TslbError) as ei:
        T.tslb_adjoint(s.handle, lam, 16, 8, g, T.HOST)  # not the handle's checkpoint interval
    assert ei.value.code == T.TSLB_ERR_INVALID
    T.tslb_adjoint(s.handle, lam, 16, 16, g, T.HOST)
    assert np.all(g == 0)  # a zero cotangent has a zero gradient
    s.close()
