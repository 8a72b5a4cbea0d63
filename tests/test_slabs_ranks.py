"""The halo exchange of the z-slab decomposition across ranks, on CPU.

exchange_halos sends each rank's bottom layer down the ring and its top layer
up it with torch.distributed point-to-point operations.  Here the ranks are
gloo processes and the slabs are CPU stand-ins that keep their layers in
numpy (no GPU): after one exchange every rank's ghost below must hold the
previous rank's top layer and its ghost above the next rank's bottom layer,
for two and three ranks (with two, both neighbours are the same rank)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2401_17074_b300.slabs import exchange_halos, ring_neighbours, split

PLANE = 24  # bytes of one packed plane of the stand-in


class FakeSlab:
    """Layers of a slab as rows of bytes; ghosts filled by halo_import."""

    def __init__(self, rank, nz):
        self.layers = [np.full(PLANE, 16 * rank + z, dtype=np.uint8) for z in range(nz)]
        self.ghost = [None, None]

    def halo_export(self, side, buf):
        buf.copy_(torch.from_numpy(self.layers[0 if side == 0 else -1]))

    def halo_import(self, side, buf):
        self.ghost[side] = buf.numpy().copy()


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nz = 3 + rank
    slab = FakeSlab(rank, nz)
    bufs = tuple(torch.zeros(PLANE, dtype=torch.uint8) for _ in range(4))
    for _ in range(2):  # two exchanges in a row reuse the buffers
        exchange_halos(slab, bufs, dist)
    lo, hi = ring_neighbours(rank, world)
    out[rank] = (int(slab.ghost[0][0]), int(slab.ghost[1][0]), 16 * lo + (3 + lo) - 1, 16 * hi)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_ring_exchange_gloo(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        got_lo, got_hi, want_lo, want_hi = out[rank]
        assert got_lo == want_lo and got_hi == want_hi, (rank, out[rank])


def test_single_rank_wraps_onto_itself():
    slab = FakeSlab(0, 4)
    bufs = tuple(torch.zeros(PLANE, dtype=torch.uint8) for _ in range(4))
    exchange_halos(slab, bufs, None)
    assert slab.ghost[0][0] == 3 and slab.ghost[1][0] == 0


def test_split_even_and_ragged():
    assert split(12, 3) == [(0, 4), (4, 8), (8, 12)]
    assert split(14, 3) == [(0, 5), (5, 10), (10, 14)]
    with pytest.raises(ValueError):
        split(8, 3)  # fewer than 3 layers per slab
