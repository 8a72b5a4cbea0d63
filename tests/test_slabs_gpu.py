"""z-slab decomposition on one GPU: a ring of halo slabs against one handle.

The lattice is cut into z slabs (TSLB_BC_HALO faces); before every step each
slab exports its bottom and top layers and imports its neighbours' into its
ghost planes (tslb_halo_export / tslb_halo_import, device copies on one
stream).  The step's arithmetic at a node does not depend on where the
lattice is cut, so the chain must reproduce the single-handle run bit for bit.
"""
import numpy as np
import pytest

import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W
from paper_2401_17074_b300.slabs import SlabChain

pytestmark = pytest.mark.gpu


def _single(dims, tau, force, bc, state, nsteps, **kw):
    s = T.Solver(dims, tau, force=force, bc=bc, kernel=T.KERNEL_FACTORED, **kw)
    s.init_moments(*state)
    s.step(nsteps)
    out = s.get_moments()
    s.close()
    return out


@pytest.mark.parametrize("overlap", [False, True], ids=["sequential", "overlapped"])
@pytest.mark.parametrize("case", ["channel-2", "channel-3-ragged", "periodic-4", "periodic-odd-3", "bf16-channel-2",
                                  "bf16-odd-2"])
def test_slab_chain_matches_single_domain(cuda_ok, case, overlap):
    # "odd": layers of an odd number of nodes (33 x 21 and 33 x 15), whose packed
    # planes end off the 16-byte boundary the second ghost plane must start on
    if case.startswith("channel") or case.startswith("bf16"):
        prm = W.channel_params(nx=33 if "odd" in case else 40, ny=17 if "odd" in case else 18,
                               nz=26 if "ragged" in case else 24)
        dims, tau, force, bc = prm["dims"], prm["tau"], prm["force"], prm["bc"]
        state = W.channel_state(prm, seed=1)
    else:
        dims, tau, force, bc = ((33, 21, 29) if "odd" in case else (34, 21, 29)), 0.62, (2e-6, -1e-6, 3e-6), (0,) * 6
        state = W.random_state(dims, seed=81)
    nslabs = int(case.split("-")[-1]) if case.split("-")[-1].isdigit() else int(case.split("-")[-2])
    kw = {}
    if case.startswith("bf16"):
        kw = dict(precision=T.BF16, u_ref=0.05, pi_ref=W.pi_reference(state))
    nsteps = 15
    ref = _single(dims, tau, force, bc, state, nsteps, **kw)
    chain = SlabChain(dims, tau, nslabs, force=force, bc=bc, overlap=overlap, **kw)
    chain.init_moments(*state)
    chain.step(nsteps)
    got = chain.get_moments()
    chain.close()
    for a, b, name in zip(got, ref, ("rho", "u", "pi")):
        assert np.array_equal(a, b), (name, np.abs(a - b).max())


def test_halo_plane_round_trip(cuda_ok):
    """A plane exported from one slab and imported as another's ghost is the
    packed [V0 | V1 | V2] layer: its size is 10 stored values per node, and
    host and device buffers give the same bytes."""
    import torch
    dims = (12, 7, 6)
    s = T.Solver(dims, 0.7, bc=(0, 0, 0, 0, T.HALO, T.HALO))
    s.init_moments(*W.random_state(dims, seed=82))
    nb = s.halo_plane_bytes()
    assert nb == 10 * 4 * 12 * 7
    host = np.zeros(nb, dtype=np.uint8)
    s.halo_export(1, host)
    dev = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    s.halo_export(1, dev)
    s.synchronize()  # the export ran on the handle's stream
    assert np.array_equal(host, dev.cpu().numpy())
    v0 = host[: 4 * 4 * 84].view(np.float32).reshape(84, 4)  # (u_x, u_y, u_z, rho - 1) of layer z = 5
    rho, u, _ = s.get_moments()
    top = slice(5 * 84, 6 * 84)
    assert np.allclose(v0[:, 3], rho[top] - 1, rtol=0, atol=1e-7)
    assert np.allclose(v0[:, 0], u[0][top], rtol=0, atol=1e-7)
    with pytest.raises(ValueError):
        s.halo_export(0, np.zeros(nb - 1, dtype=np.uint8))
    s.close()
    s2 = T.Solver(dims, 0.7)  # no halo faces
    with pytest.raises(T.TslbError) as ei:
        s2.halo_plane_bytes()
    assert ei.value.code == T.TSLB_ERR_STATE
    s2.close()


def test_halo_slab_rejects_unsupported(cuda_ok):
    dims = (12, 7, 6)
    s = T.Solver(dims, 0.7, bc=(0, 0, 0, 0, T.HALO, T.HALO))
    with pytest.raises(T.TslbError) as ei:
        s.set_force_field(np.zeros((3, 12 * 7 * 6), dtype=np.float32))
    assert ei.value.code == T.TSLB_ERR_UNSUPPORTED
    s.close()


def test_slab_chain_random_cases(cuda_ok):
    """Property-based: random lattice shapes, slab counts (ragged splits),
    y faces (periodic or bounce-back), storage types, forces and relaxation
    times; the chain must match the single handle bit for bit after a random
    number of steps."""
    from hypothesis import given, settings, HealthCheck, strategies as st

    @settings(max_examples=25, deadline=None, suppress_health_check=list(HealthCheck))
    @given(nx=st.integers(3, 45), ny=st.integers(4, 36), nslabs=st.integers(2, 5), extra=st.integers(0, 30),
           walls=st.booleans(), prec=st.sampled_from([T.FP32, T.BF16, T.FP16]), tau=st.floats(0.51, 1.5),
           steps=st.integers(1, 9), seed=st.integers(0, 10 ** 6), overlap=st.booleans())
    def run(nx, ny, nslabs, extra, walls, prec, tau, steps, seed, overlap):
        nz = 3 * nslabs + extra
        dims = (nx, ny, nz)
        bc = (0, 0, 1, 1, 0, 0) if walls else (0,) * 6
        state = W.random_state(dims, seed=seed, drho=0.005, du=0.02, dpi=2e-4)
        force = (1e-5, -2e-6, 3e-6)
        kw = {} if prec == T.FP32 else dict(precision=prec, u_ref=0.05, pi_ref=W.pi_reference(state))
        ref = _single(dims, tau, force, bc, state, steps, **kw)
        chain = SlabChain(dims, tau, nslabs, force=force, bc=bc, overlap=overlap, **kw)
        chain.init_moments(*state)
        chain.step(steps)
        got = chain.get_moments()
        chain.close()
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)

    run()


def test_split_step_states(cuda_ok):
    """tslb_step_part keeps a simple state machine: EDGES then INTERIOR; a
    whole step, an initialisation or a second EDGES while a split step is
    open, and INTERIOR with none open, are refused; a handle without halo
    faces has no split steps.  EDGES + INTERIOR equals tslb_step bit for bit
    (slab of 20 layers, so the edge and interior launches are both used)."""
    dims = (14, 9, 20)
    state = W.random_state(dims, seed=83)
    a = T.Solver(dims, 0.7, bc=(0, 0, 0, 0, T.HALO, T.HALO))
    b = T.Solver(dims, 0.7, bc=(0, 0, 0, 0, T.HALO, T.HALO))
    for s in (a, b):
        s.init_moments(*state)
    with pytest.raises(T.TslbError) as ei:
        a.step_part(T.TSLB_PART_INTERIOR)
    assert ei.value.code == T.TSLB_ERR_STATE
    a.step_part(T.TSLB_PART_EDGES)
    for bad in (lambda: a.step_part(T.TSLB_PART_EDGES), lambda: a.step(1), lambda: a.init_moments(*state)):
        with pytest.raises(T.TslbError) as ei:
            bad()
        assert ei.value.code == T.TSLB_ERR_STATE
    a.step_part(T.TSLB_PART_INTERIOR)
    b.step(1)
    for x, y in zip(a.get_moments(), b.get_moments()):
        assert np.array_equal(x, y)
    a.close()
    b.close()
    c = T.Solver(dims, 0.7)
    with pytest.raises(T.TslbError) as ei:
        c.step_part(T.TSLB_PART_EDGES)
    assert ei.value.code == T.TSLB_ERR_STATE
    c.close()


def test_step_overlapped_single_rank_ring(cuda_ok):
    """The multi-process step (slabs.step_overlapped with exchange_halos) on one
    rank: the slab is its own neighbour on both sides, the exchange runs on a
    second stream through CUDA buffers, and a lattice periodic in z as one
    halo slab must equal a plain periodic handle bit for bit."""
    import torch
    from paper_2401_17074_b300.slabs import exchange_halos, step_overlapped
    dims, tau = (37, 19, 23), 0.66
    state = W.random_state(dims, seed=84)
    force = (3e-6, 1e-6, -2e-6)
    ref = _single(dims, tau, force, (0,) * 6, state, 11)
    hs = torch.cuda.Stream()
    s = T.Solver(dims, tau, force=force, bc=(0, 0, 0, 0, T.HALO, T.HALO), halo_stream=hs.cuda_stream)
    s.init_moments(*state)
    nb = s.halo_plane_bytes()
    bufs = tuple(torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4))
    with torch.cuda.stream(hs):
        exchange_halos(s, bufs, None)  # the ghosts of the initial state
    for _ in range(11):
        step_overlapped(s, bufs, None, hs)
    got = s.get_moments()
    s.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


class _LoopbackDist:
    """A stand-in for torch.distributed with the NCCL stream semantics, on one
    GPU: world size 2 with every message coming back to this rank by its tag
    (the slab is its own ring neighbour on both sides).  A batch runs on a
    communication stream of its own that waits for the current stream when
    the batch is issued, sleeps for about a millisecond (so that an exchange
    ordered against the wrong stream reads or leaves stale planes) and then
    copies; a work's wait() makes the current stream wait for the batch."""

    isend, irecv = "send", "recv"

    class P2POp:
        def __init__(self, op, tensor, peer, tag=0):
            self.op, self.tensor, self.peer, self.tag = op, tensor, peer, tag

    def __init__(self):
        import torch
        self.torch = torch
        self.comm = torch.cuda.Stream()

    def get_world_size(self):
        return 2

    def get_rank(self):
        return 0

    def batch_isend_irecv(self, ops):
        torch = self.torch
        self.comm.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.comm):
            torch.cuda._sleep(2_000_000)
            sent = {o.tag: o.tensor for o in ops if o.op == self.isend}
            for o in ops:
                if o.op == self.irecv:
                    o.tensor.copy_(sent[o.tag])
        done = torch.cuda.Event()
        done.record(self.comm)

        class Work:
            def wait(self_):
                torch.cuda.current_stream().wait_event(done)

        return [Work() for _ in ops]


@pytest.mark.parametrize("mode", ["handle-stream", "caller-stream", "overlapped"])
def test_exchange_halos_stream_order(cuda_ok, mode):
    """exchange_halos with CUDA buffers and point-to-point operations on
    another stream (the NCCL semantics, emulated on one GPU): the exports must
    complete before the sends read the buffers and the receives before the
    imports, whether the slab runs on the handle's own stream (host waits),
    on a stream the caller gave (stream order), or with the exchange on a
    halo stream overlapping the interior update.  A lattice periodic in z as
    one halo slab must equal a plain periodic handle bit for bit."""
    import torch
    from paper_2401_17074_b300.slabs import exchange_halos, step_overlapped
    dims, tau, nsteps = (41, 17, 19), 0.71, 9
    state = W.random_state(dims, seed=85)
    force = (2e-6, -1e-6, 1e-6)
    ref = _single(dims, tau, force, (0,) * 6, state, nsteps)
    dist = _LoopbackDist()
    bc = (0, 0, 0, 0, T.HALO, T.HALO)
    st = torch.cuda.Stream()
    if mode == "handle-stream":
        s = T.Solver(dims, tau, force=force, bc=bc)
    elif mode == "caller-stream":
        s = T.Solver(dims, tau, force=force, bc=bc, stream=st.cuda_stream)
    else:
        s = T.Solver(dims, tau, force=force, bc=bc, halo_stream=st.cuda_stream)
    s.init_moments(*state)
    nb = s.halo_plane_bytes()
    bufs = tuple(torch.zeros(nb, dtype=torch.uint8, device="cuda") for _ in range(4))
    if mode == "overlapped":
        with torch.cuda.stream(st):
            exchange_halos(s, bufs, dist)
        for _ in range(nsteps):
            step_overlapped(s, bufs, dist, st)
    else:
        for _ in range(nsteps):
            if mode == "caller-stream":
                # a late export: the sends must wait for it on the slab's stream
                with torch.cuda.stream(st):
                    torch.cuda._sleep(1_000_000)
            exchange_halos(s, bufs, dist)
            s.step(1)
    got = s.get_moments()
    s.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
