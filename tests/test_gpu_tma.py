"""The 3D FP32 step's plane staging by the tensor-memory accelerator (TMA).

Where the rows of the grid are whole multiples of 16 bytes and no x or y side
is periodic, every CTA receives each plane as boxes copied by
cp.async.bulk.tensor onto an mbarrier, instead of one cp.async per cell.  The
staging mechanism must not change a bit of the result:

* TMA against the per-cell copies (PF_TMA=0 at pf_create) bit for bit: no-flux
  boxes with every (1 - A) term and a temperature gradient, Dirichlet ghost
  cells along x, Dirichlet ghost planes along z, tiles cut by the grid's edge,
  short z-chunks (PF_ZCHUNK), the overlapped upload (pf_set_fields_step), and
  z-slabs whose ghost planes sit beyond the slab (PF_BC_HALO);
* a bounded wait: with the copies left out (PF_TEST_DROP_COPIES=1, a test
  switch), the mbarrier wait runs out after about half a second, the kernel
  records it and returns, and the next synchronising call reports
  PF_ETIMEOUT; the context stays usable.
"""
import time

import numpy as np
import pytest

from paper_2303_09671_gb300 import pf
from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300.slabs import LocalSlabs

pytestmark = pytest.mark.gpu


def front_along_z(nx, ny, nz, seed, **kw):
    """random_state with its front along z instead of x (axes x and z swapped),
    so that a Dirichlet z side meets the liquid."""
    _, phi, cs, cl = wl.random_state(3, (nz, ny, nx), dx=0.5, seed=seed, **kw)
    pr, *_ = wl.random_state(3, (nx, ny, nz), dx=0.5, seed=seed, **kw)
    t = lambda a: np.ascontiguousarray(np.transpose(a, (2, 1, 0)))
    return pr, t(phi), t(cs), t(cl)


CASES = {
    "noflux_all_terms": lambda: wl.random_state(3, (64, 48, 24), dx=0.5, A=0.4, b=0.3, a=-0.3, seed=12,
                                                G_theta=0.05),
    "dirichlet_x": lambda: wl.random_state(3, (96, 40, 20), dx=0.5, A=1.5, b=0.3, seed=8,
                                           bc_lo=("noflux",) * 3, bc_hi=("dirichlet", "noflux", "noflux")),
    "dirichlet_z_planes": lambda: front_along_z(48, 32, 40, 13, A=1.5, b=0.3,
                                                bc_lo=("noflux",) * 3, bc_hi=("noflux", "noflux", "dirichlet")),
    "partial_tiles_7pt": lambda: wl.random_state(3, (36, 20, 12), dx=0.5, A=1.5, b=0.3, seed=14, lap=7),
    "partial_tiles_cubic": lambda: wl.random_state(3, (128, 17, 9), dx=0.5, A=0.4, b=0.3, seed=15,
                                                   interp="cubic"),
}


def run(pr, fields, steps, monkeypatch, tma, zchunk=None, upload_step=False):
    monkeypatch.setenv("PF_TMA", "1" if tma else "0")
    if zchunk:
        monkeypatch.setenv("PF_ZCHUNK", str(zchunk))
    else:
        monkeypatch.delenv("PF_ZCHUNK", raising=False)
    phi, cs, cl = (np.ascontiguousarray(a, dtype=np.float32) for a in fields)
    with pf.Sim(pr, "fp32") as s:
        if upload_step:
            import torch
            dev = [torch.from_numpy(a).cuda() for a in (phi, cs, cl)]
            s.set_fields_step(*dev, n=steps)
        else:
            s.set_fields(phi, cs, cl)
            s.step(steps)
        out = s.get_fields()
    return out


@pytest.mark.parametrize("case", sorted(CASES))
def test_tma_staging_equals_per_cell_copies(case, monkeypatch):
    pr, *fields = CASES[case]()
    assert pr["n"][0] * 4 % 16 == 0
    want = run(pr, fields, 6, monkeypatch, tma=False)
    got = run(pr, fields, 6, monkeypatch, tma=True)
    for a, b in zip(want, got):
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)


def test_tma_staging_short_chunks_and_overlapped_upload(monkeypatch):
    pr, *fields = CASES["noflux_all_terms"]()
    want = run(pr, fields, 4, monkeypatch, tma=False)
    for kw in (dict(zchunk=5), dict(upload_step=True)):
        got = run(pr, fields, 4, monkeypatch, tma=True, **kw)
        for a, b in zip(want, got):
            assert np.array_equal(a, b), kw


@pytest.mark.parametrize("zbc", ["noflux", "periodic"])
def test_tma_staging_of_slabs_with_ghost_planes(zbc, monkeypatch):
    """Two slabs of a 48 x 20 x 29 grid: the boxes of a slab's first and last
    planes reach its ghost planes (tensor-map planes -2 .. n_z + 1)."""
    bc = ("noflux", "noflux", zbc)
    pr, phi, cs, cl = wl.random_state(3, (48, 20, 29), dx=0.5, A=1.5, b=0.3, a=-0.3, seed=41,
                                      bc_lo=bc, bc_hi=bc)
    phi, cs, cl = (np.ascontiguousarray(a, dtype=np.float32) for a in (phi, cs, cl))
    monkeypatch.setenv("PF_TMA", "0")
    with pf.Sim(pr, "fp32") as s:
        s.set_fields(phi, cs, cl)
        s.step(8)
        want = s.get_fields()
    monkeypatch.setenv("PF_TMA", "1")
    sl = LocalSlabs(pr, "fp32", 2)
    try:
        sl.set_fields(phi, cs, cl)
        sl.step(8)
        got = sl.get_fields()
    finally:
        sl.close()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


def test_bounded_wait_reports_a_timeout(monkeypatch):
    pr, phi, cs, cl = wl.random_state(3, (64, 48, 24), dx=0.5, A=1.5, b=0.3, seed=12)
    monkeypatch.setenv("PF_TMA", "1")
    monkeypatch.setenv("PF_TEST_DROP_COPIES", "1")
    s = pf.Sim(pr, "fp32")
    monkeypatch.delenv("PF_TEST_DROP_COPIES")
    try:
        s.set_fields(phi, cs, cl)
        t0 = time.perf_counter()
        s.step(1)
        with pytest.raises(pf.PFError) as exc:
            s.sync()
        assert exc.value.code == -5      # PF_ETIMEOUT
        assert "bounded wait" in str(exc.value)
        assert time.perf_counter() - t0 < 30.0
        s.sync()                          # reported once, then cleared
    finally:
        s.close()
    # the context is still usable: a handle without the switch steps correctly
    want = run(pr, (phi, cs, cl), 2, monkeypatch, tma=False)
    got = run(pr, (phi, cs, cl), 2, monkeypatch, tma=True)
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
