"""Domain decomposition of a 3D grid along z (argument marshalling and the
exchange schedule only: every step and every reduction runs in libpf).

The explicit step's stencil reaches two cells across a face: the face fluxes
of Eqs. cs_nonvar / cl_nonvar take the phase-field rate of the cells on both
sides, and that rate takes their neighbours.  So a grid cut into slabs of whole
x-y planes advances bit for bit as the whole grid does if, before every step,
each slab imports the two planes beyond each cut from its neighbour (libpf's
PF_BC_HALO sides, pf_get_halo / pf_set_halo).  Outer z ends keep the grid's
own boundary condition; a periodic z axis makes the first and last slabs
neighbours.

* slab_extent / neighbours / slab_params: the partition and each slab's
  problem description;
* exchange: one round of point-to-point transfers between ranks (any
  torch.distributed backend: NCCL between GPUs, gloo on the CPU) -- my two
  lowest planes to the lower neighbour, my two highest to the upper one, my low
  ghosts from the lower neighbour's highest planes and my high ghosts from the
  upper neighbour's lowest;
* SlabRun: one rank's slab (a Sim with halo sides) stepped with an exchange
  before every step, and the grid's diagnostics as reductions over ranks;
* LocalSlabs: all slabs of a grid in one process on one GPU, the halos
  exchanged by device copies (the decomposition without a second GPU).

Both step by the split step of libpf (pf_step_begin / pf_step_end): the
z-chunks that read no ghost plane start first, on a stream of the handle's
own, and the exchange runs beside them; the chunks next to the cuts follow
once the ghost planes are in.  The result is the same bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

from .pf import Sim


def slab_extent(nz: int, parts: int, index: int):
    """(first plane, planes) of slab `index` of `parts`: contiguous, the first
    nz % parts slabs one plane longer."""
    if not 0 <= index < parts or parts < 1:
        raise ValueError("slab index out of range")
    base, extra = divmod(int(nz), int(parts))
    z0 = index * base + min(index, extra)
    return z0, base + (1 if index < extra else 0)


def neighbours(index: int, parts: int, periodic: bool):
    """(lower, upper) neighbour of slab `index`, None at a closed end of the
    grid; with a periodic z axis the first and last slabs are neighbours."""
    lo = index - 1 if index > 0 else (parts - 1 if periodic else None)
    hi = index + 1 if index < parts - 1 else (0 if periodic else None)
    return lo, hi


def slab_params(pr: dict, parts: int, index: int) -> dict:
    """The parameter dict of slab `index`: its own planes along z, halo sides
    where it borders another slab, the grid's boundary condition elsewhere."""
    if pr["dim"] != 3:
        raise ValueError("the decomposition is along z of a 3D grid")
    if parts == 1:
        return dict(pr)
    nx, ny, nz = (int(v) for v in pr["n"])
    z0, nzl = slab_extent(nz, parts, index)
    if nzl < 3:
        raise ValueError("every slab needs at least 3 planes")
    periodic = pr["bc_lo"][2] == "periodic"
    lo, hi = neighbours(index, parts, periodic)
    bc_lo, bc_hi = list(pr["bc_lo"]), list(pr["bc_hi"])
    bc_lo[2] = "halo" if lo is not None else pr["bc_lo"][2]
    bc_hi[2] = "halo" if hi is not None else pr["bc_hi"][2]
    return dict(pr, n=(nx, ny, nzl), bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi))


def exchange(send_lo, send_hi, recv_lo, recv_hi, lo, hi, dist, group=None):
    """One halo exchange: send_lo (my two lowest planes) to rank `lo`, send_hi
    to rank `hi`; recv_lo from `lo` (its two highest planes), recv_hi from `hi`
    (its two lowest).  A None neighbour is a closed end: nothing is sent or
    received there.  Tags keep the two directions apart where both neighbours
    are the same rank (two slabs on a periodic axis); the order of the
    operations is the same on every rank, which is all NCCL matches on."""
    P2P = dist.P2POp
    ops = []
    if lo is not None:
        ops.append(P2P(dist.isend, send_lo, lo, group, 0))
    if hi is not None:
        ops.append(P2P(dist.isend, send_hi, hi, group, 1))
    if hi is not None:
        ops.append(P2P(dist.irecv, recv_hi, hi, group, 0))
    if lo is not None:
        ops.append(P2P(dist.irecv, recv_lo, lo, group, 1))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class SlabRun:
    """Rank `rank` of `world` holds slab `rank` of the grid described by `pr`.

    step() exchanges the halos and advances one step at a time; energy(),
    solute_total() and front() return the whole grid's values (FP64 sums and
    maxima over ranks).  The handle runs on torch's current CUDA stream, which
    the NCCL transfers are ordered with."""

    def __init__(self, pr: dict, precision: str, rank: int, world: int, dist, group=None, sim=None,
                 device="cuda"):
        """sim: the slab's handle (default: a Sim of slab_params(pr, world,
        rank)); device: where the exchange buffers and reductions live (the
        GPU with NCCL, "cpu" with gloo)."""
        import torch
        self.pr, self.precision, self.rank, self.world = dict(pr), precision, rank, world
        self.dist, self.group, self.device = dist, group, device
        nz = int(pr["n"][2])
        self.z0, self.nzl = slab_extent(nz, world, rank)
        periodic = pr["bc_lo"][2] == "periodic"
        self.lo, self.hi = neighbours(rank, world, periodic) if world > 1 else (None, None)
        self.sim = sim if sim is not None else Sim(slab_params(pr, world, rank), precision)
        self.halo = world > 1
        if self.halo:
            nb = self.sim.halo_bytes()
            self.bufs = [torch.empty(nb, dtype=torch.uint8, device=device) for _ in range(4)]
        self.fresh = False

    def set_fields(self, phi, cs, cl):
        """The slab's own planes (arrays or CUDA tensors of shape (nzl, ny, nx))."""
        self.sim.set_fields(phi, cs, cl)
        self.fresh = False

    def exchange(self):
        if not self.halo:
            return
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        if self.lo is not None:
            self.sim.get_halo(0, send_lo)
        if self.hi is not None:
            self.sim.get_halo(1, send_hi)
        exchange(send_lo, send_hi, recv_lo, recv_hi, self.lo, self.hi, self.dist, self.group)
        if self.lo is not None:
            self.sim.set_halo(0, recv_lo)
        if self.hi is not None:
            self.sim.set_halo(1, recv_hi)
        self.fresh = True

    def step(self, n: int = 1, overlap: bool = True):
        """n steps, each after a halo exchange.  overlap: with a handle that
        has the split step, the exchange runs while the step's interior
        chunks do (the boundary chunks wait for it)."""
        split = overlap and self.halo and hasattr(self.sim, "step_begin")
        for _ in range(int(n)):
            if self.fresh:            # halos already in for this state
                self.sim.step(1)
            elif split:
                self.sim.step_begin()
                self.exchange()
                self.sim.step_end()
            else:
                self.exchange()
                self.sim.step(1)
            self.fresh = False

    def _reduce(self, values, op):
        import torch
        t = torch.tensor(values, dtype=torch.float64, device=self.device)
        if self.world > 1:
            self.dist.all_reduce(t, op=op, group=self.group)
        return [float(v) for v in t.cpu()]

    def energy(self) -> float:
        if not self.fresh:
            self.exchange()
        return self._reduce([self.sim.energy()], self.dist.ReduceOp.SUM)[0]

    def solute_total(self) -> float:
        return self._reduce([self.sim.solute_total()], self.dist.ReduceOp.SUM)[0]

    def front(self):
        """(x_front, c_max) of the grid: the largest crossing and concentration
        over all slabs (NaN when no slab has a crossing)."""
        xf, _, cm = self.sim.front()
        xf = -math.inf if math.isnan(xf) else xf
        xf, cm = self._reduce([xf, cm], self.dist.ReduceOp.MAX)
        return (math.nan if xf == -math.inf else xf), cm

    def get_fields(self):
        return self.sim.get_fields()

    def close(self):
        self.sim.close()


class LocalSlabs:
    """Every slab of the grid in this process, on the current GPU: the halo
    exchange is a device copy from each slab's boundary planes into its
    neighbour's ghost planes.  Stepping it is the decomposed step without a
    second GPU; the result equals the undecomposed grid's bit for bit."""

    def __init__(self, pr: dict, precision: str, parts: int):
        import torch
        if parts < 2:
            raise ValueError("LocalSlabs needs at least two slabs")
        self.pr, self.parts = dict(pr), parts
        nz = int(pr["n"][2])
        self.ext = [slab_extent(nz, parts, i) for i in range(parts)]
        periodic = pr["bc_lo"][2] == "periodic"
        self.nb = [neighbours(i, parts, periodic) for i in range(parts)]
        self.sims = [Sim(slab_params(pr, parts, i), precision) for i in range(parts)]
        self.buf = torch.empty(self.sims[0].halo_bytes(), dtype=torch.uint8, device="cuda")

    def set_fields(self, phi, cs, cl):
        """The whole grid's fields, shape (nz, ny, nx)."""
        for s, (z0, nzl) in zip(self.sims, self.ext):
            s.set_fields(*(np.ascontiguousarray(a[z0:z0 + nzl]) for a in (phi, cs, cl)))

    def exchange(self):
        for i, (lo, hi) in enumerate(self.nb):
            if hi is not None:                   # my highest planes -> upper's low ghosts
                self.sims[i].get_halo(1, self.buf)
                self.sims[hi].set_halo(0, self.buf)
            if lo is not None:                   # my lowest planes -> lower's high ghosts
                self.sims[i].get_halo(0, self.buf)
                self.sims[lo].set_halo(1, self.buf)

    def step(self, n: int = 1, overlap: bool = True):
        """n steps; overlap: every slab's interior is queued before the
        exchange, and its boundary chunks after it."""
        for _ in range(int(n)):
            if overlap:
                for s in self.sims:
                    s.step_begin()
            self.exchange()
            for s in self.sims:
                if overlap:
                    s.step_end()
                else:
                    s.step(1)

    def get_fields(self):
        parts = [s.get_fields() for s in self.sims]
        return tuple(np.concatenate([p[k] for p in parts], axis=0) for k in range(3))

    def energy(self) -> float:
        self.exchange()
        return float(sum(s.energy() for s in self.sims))

    def solute_total(self) -> float:
        return float(sum(s.solute_total() for s in self.sims))

    def close(self):
        for s in self.sims:
            s.close()
