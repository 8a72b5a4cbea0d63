"""Slab decomposition of a TSLB lattice along z.

The paper's Conclusions name the multi-GPU extension of the thread-safe
scheme as future work.  Its natural form here is a split of the lattice into
z slabs: each slab is one handle whose z faces are TSLB_BC_HALO, and each
time step needs, before it, one layer of the 10 stored moment fields from
each neighbour (the step of Eq. pushLB reaches one node in every direction).
The slabs form a ring, so the lattice stays periodic in z.

Two drivers share the same exchange pattern:

* ``SlabChain`` keeps every slab in this process, on one device and one
  stream, and moves the packed planes with device copies.  Stream order makes
  the sequence export -> import -> step correct without further
  synchronisation.  With ``overlap=True`` every step is split
  (tslb_step_part): the slabs' edge layers first, then their interiors on the
  compute stream while the exports and imports run on a second stream, which
  the library orders against the steps with events.
* ``exchange_halos`` is the multi-process form: one slab per rank, the packed
  planes sent to and received from the ring neighbours with
  ``torch.distributed`` point-to-point operations (NCCL for CUDA buffers, gloo
  for CPU buffers).  A slab is any object with ``halo_export(side, buf)`` and
  ``halo_import(side, buf)``, so the bookkeeping can run on CPU stand-ins.
"""
import contextlib

import numpy as np

from . import FP32, HALO, PERIODIC, TSLB_PART_EDGES, TSLB_PART_INTERIOR, Solver

# message tags: planes travelling up the ring (a slab's top layer to the next
# slab's lower ghost) and down it (bottom layer to the previous slab's upper ghost)
TAG_UP, TAG_DOWN = 1, 2


def split(nz, nslabs):
    """z ranges [z0, z1) of nslabs slabs covering nz layers, as even as possible."""
    if nslabs < 1 or nz < 3 * nslabs:
        raise ValueError("each slab needs at least 3 layers")
    base, extra = divmod(nz, nslabs)
    out, z = [], 0
    for s in range(nslabs):
        n = base + (1 if s < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def ring_neighbours(rank, world):
    """(rank below, rank above) in the ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def exchange_halos(slab, bufs, dist):
    """One halo exchange of this rank's slab with its ring neighbours.

    bufs = (send_lo, send_hi, recv_lo, recv_hi): buffers of one packed plane
    each (CUDA tensors with NCCL, CPU tensors with gloo).  The slab's bottom
    layer goes down the ring and its top layer up; the planes received fill
    its ghost layers below (from the rank below) and above (from the rank
    above).  With one rank the slab is its own neighbour on both sides.

    With CUDA buffers the exports and imports run on the slab's halo-copy
    stream and the point-to-point operations on PyTorch's current stream, so
    the two are ordered here: where the slab's stream is known
    (slab.halo_copy_stream, the stream or halo_stream the Solver was created
    with) the operations are issued with that stream current, so they follow
    the exports and the imports follow their completion without a host wait;
    otherwise (the handle's own stream) the host waits for the exports before
    the sends and for the receives before the imports."""
    send_lo, send_hi, recv_lo, recv_hi = bufs
    slab.halo_export(0, send_lo)
    slab.halo_export(1, send_hi)
    world = dist.get_world_size() if dist is not None else 1
    if world == 1:
        slab.halo_import(0, send_hi)
        slab.halo_import(1, send_lo)
        return
    lo, hi = ring_neighbours(dist.get_rank(), world)
    cuda = bool(getattr(send_lo, "is_cuda", False))
    ctx, sp = contextlib.nullcontext(), getattr(slab, "halo_copy_stream", None)
    if cuda:
        import torch
        if sp is not None:
            ctx = torch.cuda.stream(torch.cuda.ExternalStream(int(sp), device=send_lo.device))
        else:
            slab.synchronize()
    with ctx:
        ops = [dist.P2POp(dist.isend, send_hi, hi, tag=TAG_UP),
               dist.P2POp(dist.irecv, recv_lo, lo, tag=TAG_UP),
               dist.P2POp(dist.isend, send_lo, lo, tag=TAG_DOWN),
               dist.P2POp(dist.irecv, recv_hi, hi, tag=TAG_DOWN)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        if cuda and sp is None:
            torch.cuda.current_stream(send_lo.device).synchronize()
        slab.halo_import(0, recv_lo)
        slab.halo_import(1, recv_hi)


def step_overlapped(slab, bufs, dist, halo_stream):
    """One step of this rank's slab with its halo exchange overlapping the
    update of the slab's interior layers.

    slab: a Solver with halo faces created with halo_stream=halo_stream.cuda_stream
    (a torch.cuda.Stream).  The edge layers are advanced first; the exchange
    then runs on halo_stream (exports wait for the edges, the point-to-point
    operations are queued behind them on the same stream, imports behind
    those) while the interior layers are advanced on the slab's own stream;
    the next step waits for the imports.  The ghosts of the initial state
    must be in place before the first such step: call exchange_halos once
    after init_moments."""
    import torch
    slab.step_part(TSLB_PART_EDGES)
    with torch.cuda.stream(halo_stream):
        exchange_halos(slab, bufs, dist)
    slab.step_part(TSLB_PART_INTERIOR)


def _zslice(a, dims, z0, z1, ncomp):
    """Layers z0 .. z1-1 of a full-lattice array with ncomp components."""
    nx, ny, nz = dims
    a = np.asarray(a).reshape(ncomp, nz, ny * nx)
    return np.ascontiguousarray(a[:, z0:z1, :].reshape(ncomp, -1))


class SlabChain:
    """A lattice periodic in z, split into z slabs that all live in this process.

    Every slab is a Solver with halo z faces on the same device and the same
    stream; ``step`` exchanges the boundary layers through device buffers
    before every step.  The result equals a single-handle run of the whole
    lattice (the step's arithmetic at a node does not depend on where the
    lattice is cut).  bc gives the x and y faces (the z faces must be periodic).
    """

    def __init__(self, dims, tau, nslabs, force=(0.0, 0.0, 0.0), bc=(0,) * 6, precision=FP32, u_ref=0.05,
                 pi_ref=1e-3, device=0, overlap=False):
        import torch
        if bc[4] != PERIODIC or bc[5] != PERIODIC:
            raise ValueError("a slab chain is periodic in z")
        self.dims = tuple(int(d) for d in dims)
        self.ranges = split(self.dims[2], nslabs)
        self.stream = torch.cuda.Stream(device=device)
        self.overlap = bool(overlap)
        self.halo_stream = torch.cuda.Stream(device=device) if self.overlap else None
        hs = self.halo_stream.cuda_stream if self.overlap else None
        sbc = tuple(bc[:4]) + (HALO, HALO)
        self.slabs = [Solver((self.dims[0], self.dims[1], z1 - z0), tau, force=force, bc=sbc, precision=precision,
                             u_ref=u_ref, pi_ref=pi_ref, device=device, stream=self.stream.cuda_stream,
                             halo_stream=hs)
                      for z0, z1 in self.ranges]
        nb = self.slabs[0].halo_plane_bytes()
        self.bufs = [[torch.empty(nb, dtype=torch.uint8, device="cuda:%d" % device) for _ in range(2)]
                     for _ in self.slabs]

    def close(self):
        for s in self.slabs:
            s.close()

    def init_moments(self, rho, u, pi=None):
        for s, (z0, z1) in zip(self.slabs, self.ranges):
            s.init_moments(_zslice(rho, self.dims, z0, z1, 1).reshape(-1), _zslice(u, self.dims, z0, z1, 3),
                           None if pi is None else _zslice(pi, self.dims, z0, z1, 6))
        if self.overlap:
            # an overlapped step exchanges the layers of the state it produces,
            # so the ghosts of the initial state are filled here
            self.exchange()

    def exchange(self):
        n = len(self.slabs)
        for s, slab in enumerate(self.slabs):
            slab.halo_export(0, self.bufs[s][0])
            slab.halo_export(1, self.bufs[s][1])
        for s in range(n):
            self.slabs[(s + 1) % n].halo_import(0, self.bufs[s][1])
            self.slabs[(s - 1) % n].halo_import(1, self.bufs[s][0])

    def step(self, n=1):
        for _ in range(int(n)):
            if self.overlap:
                # the edges need the ghosts of this step's state; the exchange of
                # the new edge layers then overlaps the interiors
                for slab in self.slabs:
                    slab.step_part(TSLB_PART_EDGES)
                self.exchange()
                for slab in self.slabs:
                    slab.step_part(TSLB_PART_INTERIOR)
            else:
                self.exchange()
                for slab in self.slabs:
                    slab.step(1)

    def get_moments(self):
        nx, ny, nz = self.dims
        rho = np.zeros((nz, ny * nx))
        u = np.zeros((3, nz, ny * nx))
        pi = np.zeros((6, nz, ny * nx))
        for s, (z0, z1) in zip(self.slabs, self.ranges):
            r, uu, p = s.get_moments()
            rho[z0:z1] = r.reshape(z1 - z0, -1)
            u[:, z0:z1] = uu.reshape(3, z1 - z0, -1)
            pi[:, z0:z1] = p.reshape(6, z1 - z0, -1)
        return rho.reshape(-1), u.reshape(3, -1), pi.reshape(6, -1)
