"""The z-slab decomposition on one GPU: every slab of the grid in one process
(LocalSlabs), the two ghost planes per cut exchanged by device copies before
every step, against the undecomposed grid: the fields bit for bit, the free
energy and solute totals summed over the slabs to rounding.  FP32 and FP64,
no-flux and periodic z, two and three (uneven) slabs."""
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
