"""The z-slab decomposition's host side on the CPU: the partition, the
neighbours (closed and periodic z), and SlabRun's halo exchange and reductions
on 2 and 3 gloo ranks, against a NumPy reference.  Each rank's slab is a
stand-in with the handle's halo interface (two planes per side, exported and
imported through the exchange buffers) and a five-point z stencil whose
weights differ on every tap, so a ghost plane taken from the wrong side, the
wrong neighbour or in the wrong order changes the result."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_09671_gb300 import slabs  # noqa: E402

W = np.array([1.0, 2.0, 3.0, 5.0, 7.0]) / 18.0      # taps z-2 .. z+2


def reference_step(a, periodic):
    """The stencil on the whole grid: periodic wrap or mirror ghosts (the
    library's no-flux ghosts: plane -1 = plane 0, -2 = 1)."""
    nz = a.shape[0]
    out = np.zeros_like(a)
    for z in range(nz):
        for k, w in zip(range(-2, 3), W):
            zz = z + k
            if periodic:
                zz %= nz
            elif zz < 0:
                zz = -zz - 1
            elif zz >= nz:
                zz = 2 * nz - 1 - zz
            out[z] += w * a[zz]
    return out


class FakeSlab:
    """A slab with the halo interface of pf.Sim: own planes plus two ghost
    planes per side; halo sides must be imported before each step.  Its split
    step (step_begin / step_end) computes the interior planes from its own
    planes alone before any ghost is in, and the planes next to the sides in
    step_end, as the library's split step does."""

    def __init__(self, own, halo_lo, halo_hi):
        self.own = own.copy()
        self.halo = (halo_lo, halo_hi)
        self.ghost = [None, None]
        self.interior = None     # an open split step's interior planes
        self.splits = 0          # split steps taken

    def halo_bytes(self):
        return 2 * self.own[0].size * 8

    def get_halo(self, side, buf):
        planes = self.own[:2] if side == 0 else self.own[-2:]
        buf.view(torch.float64).copy_(torch.from_numpy(np.ascontiguousarray(planes).ravel()))

    def set_halo(self, side, buf):
        self.ghost[side] = buf.view(torch.float64).numpy().reshape((2,) + self.own.shape[1:]).copy()

    def _extended(self):
        lo = self.ghost[0] if self.halo[0] else self.own[1::-1]     # mirror: planes 1, 0
        hi = self.ghost[1] if self.halo[1] else self.own[:-3:-1]    # mirror: planes nz-1, nz-2
        assert lo is not None and hi is not None, "halo not imported"
        return np.concatenate([lo, self.own, hi])

    def step(self, n):
        assert n == 1 and self.interior is None
        ext = self._extended()
        self.own = sum(w * ext[k:k + self.own.shape[0]] for k, w in enumerate(W))
        self.ghost = [None, None]

    def step_begin(self):
        assert self.interior is None
        nz = self.own.shape[0]
        # planes 2 .. nz-3 read planes 0 .. nz-1 only
        self.interior = sum(w * self.own[k:k + nz - 4] for k, w in enumerate(W))

    def step_end(self):
        assert self.interior is not None, "no split step open"
        ext = self._extended()
        nz = self.own.shape[0]
        new = np.empty_like(self.own)
        new[2:nz - 2] = self.interior
        for z in (0, 1, nz - 2, nz - 1):
            new[z] = sum(w * ext[z + k] for k, w in enumerate(W))
        self.own = new
        self.ghost = [None, None]
        self.interior = None
        self.splits += 1

    def energy(self):
        assert all(g is not None for g, h in zip(self.ghost, self.halo) if h), "halo not imported"
        return float(self.own.sum())

    def solute_total(self):
        return float((self.own ** 2).sum())

    def front(self):
        return float(self.own.max()), 0.0, float((self.own ** 2).max())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, periodic, overlap, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz, ny, nx = 13, 3, 4
        a = np.random.default_rng(5).standard_normal((nz, ny, nx))
        bc = "periodic" if periodic else "noflux"
        pr = dict(dim=3, n=(nx, ny, nz), bc_lo=("noflux", "noflux", bc), bc_hi=("noflux", "noflux", bc))
        z0, nzl = slabs.slab_extent(nz, world, rank)
        sp = slabs.slab_params(pr, world, rank)
        fake = FakeSlab(a[z0:z0 + nzl], sp["bc_lo"][2] == "halo", sp["bc_hi"][2] == "halo")
        run = slabs.SlabRun(pr, "fp64", rank, world, dist, sim=fake, device="cpu")
        E = run.energy()
        run.step(4, overlap=overlap)
        S = run.solute_total()
        fmax, cmax = run.front()
        out[rank] = (z0, fake.own.copy(), E, S, fmax, cmax, fake.splits)
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("overlap", [True, False])
def test_slab_run_exchange_matches_whole_grid(world, periodic, overlap):
    """Four steps after an energy call (which imports the halos, so the first
    step is a plain one): with overlap the other three are split steps whose
    interior is computed before the exchange."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, periodic, overlap, out), nprocs=world, join=True)
        res = dict(out)
    nz, ny, nx = 13, 3, 4
    a = np.random.default_rng(5).standard_normal((nz, ny, nx))
    ref = a.copy()
    for _ in range(4):
        ref = reference_step(ref, periodic)
    got = np.concatenate([res[r][1] for r in range(world)])
    assert np.allclose(got, ref, rtol=0, atol=1e-13)
    for r in range(world):
        assert res[r][2] == pytest.approx(a.sum(), rel=1e-13)
        assert res[r][3] == pytest.approx((ref ** 2).sum(), rel=1e-12)
        assert res[r][4] == ref.max() and res[r][5] == (ref ** 2).max()
        assert res[r][6] == (3 if overlap else 0)


def test_partition_and_neighbours():
    assert [slabs.slab_extent(10, 3, i) for i in range(3)] == [(0, 4), (4, 3), (7, 3)]
    assert sum(slabs.slab_extent(256, 8, i)[1] for i in range(8)) == 256
    assert slabs.neighbours(0, 3, False) == (None, 1) and slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 3, True) == (2, 1) and slabs.neighbours(2, 3, True) == (1, 0)
    assert slabs.neighbours(0, 2, True) == (1, 1)
    pr = dict(dim=3, n=(8, 8, 20), bc_lo=("noflux", "periodic", "noflux"), bc_hi=("noflux", "periodic", "dirichlet"))
    s0, s1 = slabs.slab_params(pr, 2, 0), slabs.slab_params(pr, 2, 1)
    assert s0["n"] == (8, 8, 10) and s0["bc_lo"][2] == "noflux" and s0["bc_hi"][2] == "halo"
    assert s1["bc_lo"][2] == "halo" and s1["bc_hi"][2] == "dirichlet"
    with pytest.raises(ValueError):
        slabs.slab_params(dict(pr, n=(8, 8, 5)), 2, 1)      # 3 + 2 planes
