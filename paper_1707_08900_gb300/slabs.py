"""Domain decomposition of a periodic box into z-slabs with halo exchange.

The paper names splitting the grid over several GPUs as the way to larger
problems (Sect. 7): each device owns part of the domain and the ghost zones
at the cuts carry the neighbours' values.  Here the box is cut along z into
slabs; each slab is a solver context created with bc_z = "exchange", which
keeps three ghost planes below and above its interior and leaves them to the
caller.  Before every substep the three boundary planes of every field move
to the neighbouring slabs (one exchange per substep for the 55-point form).

* exchange(slab, rank, world, dist): one rank's part of an exchange over a
  torch.distributed process group (one slab per rank; NCCL for device
  buffers, gloo for host buffers).  Sends are posted before receives in the
  same order on every rank (side 1 to the upper neighbour, then side 0 to
  the lower one; receive from the lower neighbour into side 0, then from the
  upper one into side 1), so with two ranks, where both neighbours are the
  same rank, the two messages cannot be swapped.
* Slabs: every slab on one GPU (the ranks emulated: a message is a
  device-to-device copy between two contexts), the same schedule.

A slab object provides pack(side) -> message, empty_message(),
unpack(side, message) and substep(s, dt); SolverSlab wraps a context.
"""
import numpy as np

from . import gbfd

GZ = 3  # ghost planes per side


def split(nz, nslabs):
    """Plane ranges [(z0, z1)] of nslabs slabs as equal as possible."""
    cuts = [round(i * nz / nslabs) for i in range(nslabs + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


def exchange(slab, rank, world, dist=None, group=None):
    """This rank's part of one halo exchange (slabs ordered along z,
    periodic).  world == 1: the slab is its own neighbour on both sides."""
    send1 = slab.pack(1)
    send0 = slab.pack(0)
    if world == 1:
        slab.unpack(0, send1)
        slab.unpack(1, send0)
        return
    lo, hi = (rank - 1) % world, (rank + 1) % world
    recv0 = slab.empty_message()
    recv1 = slab.empty_message()
    reqs = [dist.isend(send1, hi, group=group, tag=0), dist.isend(send0, lo, group=group, tag=1),
            dist.irecv(recv0, lo, group=group, tag=0), dist.irecv(recv1, hi, group=group, tag=1)]
    for r in reqs:
        r.wait()
    slab.unpack(0, recv0)
    slab.unpack(1, recv1)


class SolverSlab:
    """One z-slab as a solver context (bc_z = "exchange"): the slab's nz
    planes of a box of z length lz_global split over nz_global planes."""

    def __init__(self, shape, nz_global, lengths, **kw):
        import torch
        nz, ny, nx = shape
        lx, ly, lz = lengths
        self.torch = torch
        self.solver = gbfd.Solver(shape, lengths=(lx, ly, lz * nz / nz_global), bc_z="exchange",
                                  **kw)
        self.nbytes = load_halo_bytes(self.solver)
        dev = self.solver.device
        self.msg = [torch.empty(self.nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]

    def pack(self, side):
        gbfd._check(gbfd.load().gbfd_halo_pack(self.solver.ctx, side,
                                               gbfd._VP(self.msg[side].data_ptr())),
                    self.solver.ctx)
        return self.msg[side]

    def empty_message(self):
        return self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.solver.device)

    def unpack(self, side, msg):
        gbfd._check(gbfd.load().gbfd_halo_unpack(self.solver.ctx, side, gbfd._VP(msg.data_ptr())),
                    self.solver.ctx)

    def substep(self, s, dt):
        self.solver.substep(s, dt)

    def close(self):
        self.solver.close()


def load_halo_bytes(solver):
    n = gbfd.load().gbfd_halo_bytes(solver.ctx)
    if n == 0:
        raise gbfd.GbfdError(5, "not an exchange context")
    return n


class Slabs:
    """A periodic box split into nslabs z-slabs on one GPU (ranks emulated).
    Same state interface as gbfd.Solver (55-point form)."""

    def __init__(self, shape, nslabs, lengths=(2 * np.pi,) * 3, **kw):
        self.shape = tuple(shape)
        nz = shape[0]
        self.bounds = split(nz, nslabs)
        self.slabs = [SolverSlab((z1 - z0,) + self.shape[1:], nz, lengths, **kw)
                      for z0, z1 in self.bounds]
        self._fresh = False

    def set_state(self, st):
        for (z0, z1), sl in zip(self.bounds, self.slabs):
            sl.solver.set_state(np.ascontiguousarray(st[:, z0:z1]))

    def get_state(self, fp64=True):
        return np.concatenate([sl.solver.get_state(fp64=fp64) for sl in self.slabs], axis=1)

    def exchange(self):
        """Every slab's ghost planes from its neighbours (device copies: each
        slab's unpack reads the neighbour's packed message directly)."""
        k = len(self.slabs)
        for sl in self.slabs:
            sl.pack(0)
            sl.pack(1)
        for i, sl in enumerate(self.slabs):
            sl.unpack(0, self.slabs[(i - 1) % k].msg[1])
            sl.unpack(1, self.slabs[(i + 1) % k].msg[0])

    def rk3_step(self, dt, nsteps=1):
        for _ in range(nsteps):
            for s in range(3):
                self.exchange()
                for sl in self.slabs:
                    sl.substep(s, dt)

    def sync(self):
        for sl in self.slabs:
            sl.solver.sync()

    def close(self):
        for sl in self.slabs:
            sl.close()
