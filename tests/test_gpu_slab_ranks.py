"""The decomposition across processes: two ranks, each its own process with
its own slab handle on the GPU, stepping with the real kernels and exchanging
the two ghost planes per cut before every step through torch.distributed
(gloo, host buffers: pf_get_halo / pf_set_halo with where = PF_HOST).  No
kernel waits on the other rank: every exchange happens on the host between
steps.  The gathered fields equal the undecomposed grid's bit for bit, and the
grid diagnostics reduced over the ranks equal the grid's to rounding."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

GRID = (40, 17, 23)


def _problem(zbc):
    sys.path.insert(0, ROOT)
    from paper_2303_09671_gb300 import workloads as wl
    bc = ("noflux", "periodic", zbc)
    return wl.random_state(3, GRID, dx=0.5, A=1.5, b=0.3, a=-0.3, seed=61, bc_lo=bc, bc_hi=bc)


def _rank(rank, world, port, zbc, precision, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2303_09671_gb300.slabs import SlabRun
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr, phi, cs, cl = _problem(zbc)
        dt = np.float64 if precision == "fp64" else np.float32
        run = SlabRun(pr, precision, rank, world, dist, device="cpu")
        sl = slice(run.z0, run.z0 + run.nzl)
        run.set_fields(*(np.ascontiguousarray(a[sl], dtype=dt) for a in (phi, cs, cl)))
        E0, S0 = run.energy(), run.solute_total()
        run.step(10)
        E1, S1 = run.energy(), run.solute_total()
        xf, cm = run.front()
        out[rank] = (run.z0, run.get_fields(), (E0, S0, E1, S1, xf, cm))
        run.close()
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("zbc", ["noflux", "periodic"])
def test_two_rank_processes_equal_the_whole_grid(precision, zbc):
    import torch.multiprocessing as mp
    from paper_2303_09671_gb300.pf import Sim
    pr, phi, cs, cl = _problem(zbc)
    dt = np.float64 if precision == "fp64" else np.float32
    with Sim(pr, precision) as s:
        s.set_fields(*(np.asarray(a, dtype=dt) for a in (phi, cs, cl)))
        E0, S0 = s.energy(), s.solute_total()
        s.step(10)
        E1, S1 = s.energy(), s.solute_total()
        xf, _, cm = s.front()
        want = s.get_fields()
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, zbc, precision, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    got = [np.concatenate([res[r][1][k] for r in (0, 1)], axis=0) for k in range(3)]
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    for r in (0, 1):
        e0, s0, e1, s1, gxf, gcm = res[r][2]
        assert e0 == pytest.approx(E0, rel=1e-12) and e1 == pytest.approx(E1, rel=1e-12)
        assert s0 == pytest.approx(S0, rel=1e-13) and s1 == pytest.approx(S1, rel=1e-13)
        assert gxf == pytest.approx(xf, rel=1e-14) and gcm == cm
