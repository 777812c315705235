"""Pin of the oracle's slab substep (a z-slab of a periodic domain split
along z, ghost planes holding the neighbouring slabs' planes; the domain
decomposition of Sect. 7) and the CPU check of the product's halo-exchange
schedule with two gloo ranks.

Pin: the slabs of a periodic box, their ghost planes copied from the
neighbours before every substep, reproduce the periodic oracle on the whole
box bit for bit: every interior point reads the same stencil values in the
same order as in the undivided box."""
import os

import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import inputs

G = fd.GZ_WALL


def _slab_bounds(nz, k):
    cuts = [round(i * nz / k) for i in range(k + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


def _fill_from_neighbours(exts):
    """Ghost planes of each slab from its neighbours' interior planes."""
    k = len(exts)
    for i, e in enumerate(exts):
        lo, hi = exts[(i - 1) % k], exts[(i + 1) % k]
        e[:, :G] = lo[:, lo.shape[1] - 2 * G:lo.shape[1] - G]
        e[:, e.shape[1] - G:] = hi[:, G:2 * G]


@pytest.mark.parametrize("nslabs", [2, 3])
def test_slabs_reproduce_the_periodic_box_bitwise(nslabs):
    nz, ny, nx = 27, 12, 16
    lz = 2.5
    st = inputs.spectrum((nz, ny, nx), 4, mach=0.3, lnrho_rms=0.05)
    g = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, lz)
    ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
    dt = fd.cfl_dt(st, g, ph, 0.4)
    ref = fd.rk3_step(st, dt, g, ph, nsteps=2)
    bounds = _slab_bounds(nz, nslabs)
    h = lz / nz
    exts, ws, grids = [], [], []
    for z0, z1 in bounds:
        e = np.zeros((5, z1 - z0 + 2 * G, ny, nx))
        e[:, G:G + z1 - z0] = st[:, z0:z1]
        exts.append(e)
        ws.append(np.zeros_like(e))
        grids.append(fd.Grid(nx, ny, z1 - z0, 2 * np.pi, 2 * np.pi, h * (z1 - z0)))
    for _ in range(2):
        for s in range(3):
            _fill_from_neighbours(exts)
            for i in range(nslabs):
                exts[i], ws[i] = fd.substep_slab(exts[i], ws[i], s, dt, grids[i], ph)
    got = np.concatenate([e[:, G:e.shape[1] - G] for e in exts], axis=1)
    assert np.array_equal(got, ref)
    assert np.abs(got - st).max() > 1e-3


class OracleSlab:
    """A slab held by one rank with the oracle doing the substeps: the same
    pack / unpack / substep interface as the solver's slab contexts
    (test infrastructure)."""

    def __init__(self, st_slab, nz_global, grid_global, phys):
        import torch
        self.torch = torch
        nf, nzl, ny, nx = st_slab.shape
        self.ext = np.zeros((nf, nzl + 2 * G, ny, nx))
        self.ext[:, G:G + nzl] = st_slab
        self.w = np.zeros_like(self.ext)
        h = grid_global.lz / nz_global
        self.grid = fd.Grid(nx, ny, nzl, grid_global.lx, grid_global.ly, h * nzl)
        self.phys = phys

    def pack(self, side):
        e = self.ext
        planes = e[:, G:2 * G] if side == 0 else e[:, e.shape[1] - 2 * G:e.shape[1] - G]
        return self.torch.from_numpy(np.ascontiguousarray(planes))

    def empty_message(self):
        nf, _, ny, nx = self.ext.shape
        return self.torch.zeros((nf, G, ny, nx), dtype=self.torch.float64)

    def unpack(self, side, msg):
        e = self.ext
        if side == 0:
            e[:, :G] = msg.numpy()
        else:
            e[:, e.shape[1] - G:] = msg.numpy()

    def substep(self, s, dt):
        self.ext, self.w = fd.substep_slab(self.ext, self.w, s, dt, self.grid, self.phys)

    def interior(self):
        return self.ext[:, G:self.ext.shape[1] - G]


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1707_08900_gb300 import slabs
        nz, ny, nx = 22, 8, 12
        st = inputs.spectrum((nz, ny, nx), 6, mach=0.3, lnrho_rms=0.05)
        g = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, 3.0)
        ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
        dt = fd.cfl_dt(st, g, ph, 0.4)
        z0, z1 = slabs.split(nz, world)[rank]
        slab = OracleSlab(st[:, z0:z1], nz, g, ph)
        for _ in range(2):
            for s in range(3):
                slabs.exchange(slab, rank, world, dist)
                slab.substep(s, dt)
        parts = [None] * world
        dist.all_gather_object(parts, slab.interior())
        if rank == 0:
            got = np.concatenate(parts, axis=1)
            ref = fd.rk3_step(st, dt, g, ph, nsteps=2)
            np.save(result_path, np.array([float(np.array_equal(got, ref)),
                                           float(np.abs(got - ref).max())]))
    finally:
        dist.destroy_process_group()


def test_halo_exchange_schedule_on_two_gloo_ranks(tmp_path):
    """The product's exchange schedule (paper_1707_08900_gb300.slabs.exchange)
    between two gloo ranks, each stepping its slab with the oracle: the
    gathered result is the periodic oracle on the whole box, bit for bit
    (with two ranks both neighbours are the same rank, so the two messages
    must not be mixed up)."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    out = str(tmp_path / "res.npy")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True,
                       start_method="spawn")
    equal, maxdiff = np.load(out)
    assert equal == 1.0, maxdiff
