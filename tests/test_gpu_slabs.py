"""The z-slab decomposition on one GPU: every slab of the grid in one process
(LocalSlabs), the two ghost planes per cut exchanged by device copies before
every step, against the undecomposed grid: the fields bit for bit, the free
energy and solute totals summed over the slabs to rounding.  FP32 and FP64,
no-flux and periodic z, two and three (uneven) slabs.  The split step
(pf_step_begin / pf_step_end: the chunks that read no ghost plane before the
exchange, the others after it) against the plain step, and its rules."""
import numpy as np
import pytest

from paper_2303_09671_gb300 import pf
from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300.slabs import LocalSlabs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("zbc,parts", [("noflux", 2), ("noflux", 3), ("periodic", 2), ("periodic", 3)])
def test_slabs_equal_the_whole_grid(precision, zbc, parts):
    bc = ("noflux", "periodic", zbc)
    pr, phi, cs, cl = wl.random_state(3, (45, 19, 29), dx=0.5, A=1.5, b=0.3, a=-0.3, seed=41,
                                      bc_lo=bc, bc_hi=bc)
    dt = np.float64 if precision == "fp64" else np.float32
    phi, cs, cl = (np.ascontiguousarray(a, dtype=dt) for a in (phi, cs, cl))
    with pf.Sim(pr, precision) as s:
        s.set_fields(phi, cs, cl)
        E0, S0 = s.energy(), s.solute_total()
        s.step(12)
        want = s.get_fields()
        E1, S1 = s.energy(), s.solute_total()
    sl = LocalSlabs(pr, precision, parts)
    try:
        sl.set_fields(phi, cs, cl)
        assert sl.energy() == pytest.approx(E0, rel=1e-12)
        assert sl.solute_total() == pytest.approx(S0, rel=1e-13)
        sl.step(12)
        got = sl.get_fields()
        for a, b in zip(want, got):
            assert np.array_equal(a, b)
        assert sl.energy() == pytest.approx(E1, rel=1e-12)
        assert sl.solute_total() == pytest.approx(S1, rel=1e-13)
    finally:
        sl.close()


def test_halo_rules():
    """A slab steps one step at a time and only with its halos imported; a
    side that is not a halo side has none to import or export; a slab cannot
    upload and step in one call."""
    import torch
    bc = ("noflux", "noflux", "noflux")
    pr, phi, cs, cl = wl.random_state(3, (40, 16, 12), dx=0.5, A=1.5, b=0.3, seed=42, bc_lo=bc, bc_hi=bc)
    sp = dict(pr, bc_hi=("noflux", "noflux", "halo"))
    with pf.Sim(sp, "fp64") as s:
        s.set_fields(phi, cs, cl)
        buf = torch.zeros(s.halo_bytes(), dtype=torch.uint8, device="cuda")
        assert s.halo_bytes() == 3 * 2 * 40 * 16 * 8
        with pytest.raises(pf.PFError, match="halo not imported"):
            s.step(1)
        with pytest.raises(pf.PFError, match="halo not imported"):
            s.energy()
        with pytest.raises(pf.PFError, match="not a halo side"):
            s.get_halo(0, buf)
        s.get_halo(1, buf)
        s.set_halo(1, buf)
        with pytest.raises(pf.PFError, match="one step at a time"):
            s.step(2)
        s.step(1)
        with pytest.raises(pf.PFError, match="halo not imported"):
            s.step(1)
        with pytest.raises(pf.PFError, match="halo sides"):
            s.set_fields_step(phi, cs, cl, n=1)
        # host buffers: the exported planes are the top two planes of the state
        s.set_fields(phi, cs, cl)
        hb = np.zeros(s.halo_bytes() // 8)
        s.get_halo(1, hb)
        assert np.array_equal(hb[: 2 * 40 * 16].reshape(2, 16, 40), phi[-2:])


SPLIT_GRIDS = {
    # rows of 48 FP32 words and no periodic x/y side: TMA-staged planes
    "tma": dict(n=(48, 20, 29), bc_xy=("noflux", "noflux")),
    # periodic y and rows of 45 words: per-cell copies
    "copies": dict(n=(45, 19, 29), bc_xy=("noflux", "periodic")),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("grid", sorted(SPLIT_GRIDS))
@pytest.mark.parametrize("zbc,parts,zchunk", [("noflux", 2, 3), ("periodic", 3, 2), ("periodic", 2, 4),
                                              ("noflux", 3, 0)])
def test_split_step_slabs_equal_the_whole_grid(precision, grid, zbc, parts, zchunk, monkeypatch):
    """LocalSlabs stepped by the split step (every slab's interior chunks
    queued before the exchange, the chunks next to the cuts after it) equals
    the undecomposed grid bit for bit.  Short z-chunks give each slab several
    interior chunks; zchunk 0 is the automatic choice."""
    g = SPLIT_GRIDS[grid]
    bc = g["bc_xy"] + (zbc,)
    pr, phi, cs, cl = wl.random_state(3, g["n"], dx=0.5, A=1.5, b=0.3, a=-0.3, seed=43, bc_lo=bc, bc_hi=bc)
    dt = np.float64 if precision == "fp64" else np.float32
    phi, cs, cl = (np.ascontiguousarray(a, dtype=dt) for a in (phi, cs, cl))
    with pf.Sim(pr, precision) as s:
        s.set_fields(phi, cs, cl)
        s.step(10)
        want = s.get_fields()
    if zchunk:
        monkeypatch.setenv("PF_ZCHUNK", str(zchunk))
    sl = LocalSlabs(pr, precision, parts)
    try:
        sl.set_fields(phi, cs, cl)
        sl.step(10, overlap=True)
        got = sl.get_fields()
    finally:
        sl.close()
    for a, b in zip(want, got):
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)


@pytest.mark.parametrize("zbc", ["noflux", "periodic"])
def test_split_step_of_a_whole_grid_equals_step(zbc, monkeypatch):
    """Without halo sides the split step is still the step: the interior
    chunks, then the first and last chunks (a periodic z wraps inside them)."""
    bc = ("noflux", "noflux", zbc)
    pr, phi, cs, cl = wl.random_state(3, (64, 24, 23), dx=0.5, A=0.4, b=0.3, seed=44, bc_lo=bc, bc_hi=bc,
                                      G_theta=0.05)
    phi, cs, cl = (np.ascontiguousarray(a, dtype=np.float32) for a in (phi, cs, cl))
    monkeypatch.setenv("PF_ZCHUNK", "4")
    with pf.Sim(pr, "fp32") as s:
        s.set_fields(phi, cs, cl)
        s.step(6)
        want = s.get_fields()
    with pf.Sim(pr, "fp32") as s:
        s.set_fields(phi, cs, cl)
        for _ in range(6):
            s.step_begin()
            s.step_end()
        assert s.clock == (6, 0)
        got = s.get_fields()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


def test_split_step_rules(monkeypatch):
    """Between pf_step_begin and pf_step_end the calls that change the state
    or the clock are refused and those that read it are allowed; pf_step_end
    without a halo import is refused and leaves the split open; the split
    step needs a 3D grid."""
    import torch
    monkeypatch.setenv("PF_ZCHUNK", "3")
    bc = ("noflux", "noflux", "noflux")
    pr, phi, cs, cl = wl.random_state(3, (40, 16, 14), dx=0.5, A=1.5, b=0.3, seed=45, bc_lo=bc, bc_hi=bc)
    phi, cs, cl = (np.ascontiguousarray(a, dtype=np.float64) for a in (phi, cs, cl))
    sp = dict(pr, bc_hi=("noflux", "noflux", "halo"))
    with pf.Sim(sp, "fp64") as s, pf.Sim(sp, "fp64") as ref:
        buf = torch.zeros(s.halo_bytes(), dtype=torch.uint8, device="cuda")
        for h in (s, ref):
            h.set_fields(phi, cs, cl)
        ref.get_halo(1, buf)
        ref.set_halo(1, buf)
        ref.step(1)
        want = ref.get_fields()
        with pytest.raises(pf.PFError, match="no split step is open"):
            s.step_end()
        s.step_begin()
        with pytest.raises(pf.PFError, match="split step is open"):
            s.step_begin()
        with pytest.raises(pf.PFError, match="split step is open"):
            s.step(1)
        with pytest.raises(pf.PFError, match="split step is open"):
            s.set_fields(phi, cs, cl)
        with pytest.raises(pf.PFError, match="halo not imported"):
            s.step_end()
        before = s.get_fields()                  # reading the current state is allowed
        assert np.array_equal(before[0], phi)
        s.get_halo(1, buf)
        s.set_halo(1, buf)
        s.energy()
        s.step_end()                             # the split was still open
        assert s.clock == (1, 0)
        got = s.get_fields()
        for a, b in zip(want, got):
            assert np.array_equal(a, b)
    pr2, phi2, cs2, cl2 = wl.random_state(2, (32, 16), dx=0.5, seed=46)
    with pf.Sim(pr2, "fp32") as s2:
        with pytest.raises(pf.PFError, match="3D grid"):
            s2.step_begin()
