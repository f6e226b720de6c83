"""pf_energy_solute_noalloc: the allocation-free energy/solute reduction, for
callers that cannot allocate device memory (their device memory is held by
another allocator, they run on a path that must not block or fail on an
allocation, or they have no pf_handle), checked against pf_energy and
pf_solute_total on two calls in a row.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300 import pf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,maker", [
    ("fp64", lambda: wl.random_state(3, (37, 19, 13), A=1.5, b=0.3, seed=7)),
    ("fp64", lambda: wl.pulled_front_1d(N=300, V=0.1, A=1.0, b=1.0)),
    ("fp32", lambda: wl.perturbed_front_2d(nx=96, ny=64, front=30, A=1.5, b=0.3)),
])
def test_noalloc_matches_handle_reductions(precision, maker):
    import torch
    pr, phi, cs, cl = maker()
    dt = torch.float64 if precision == "fp64" else torch.float32
    npdt = np.float64 if precision == "fp64" else np.float32
    phi, cs, cl = (np.asarray(a, dtype=npdt) for a in (phi, cs, cl))
    with pf.Sim(pr, precision) as s:
        s.set_fields(phi, cs, cl)
        s.step(3)
        E_ref, S_ref = s.energy(), s.solute_total()
        fields = s.get_fields()
        step, shifts = s.clock
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    for _ in range(2):       # the shared scratch array is reused by the second call
        out.fill_(float("nan"))
        pf.energy_solute_noalloc(pr, *dev, out, precision=precision, step=step, shifts=shifts)
        torch.cuda.synchronize()
        E, S = out.cpu().numpy()
        assert abs(E - E_ref) <= tol * abs(E_ref), (E, E_ref)
        assert abs(S - S_ref) <= tol * abs(S_ref), (S, S_ref)


def test_noalloc_rejects_invalid_sizes():
    import torch
    pr, phi, cs, cl = wl.random_state(2, (8, 8))
    t = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(t.data_ptr())

    def c_call(pr_, **over):
        # straight through the C ABI with real device pointers: the entry point's
        # own checks, whatever the binding checks first
        g, b, p = pf.make_structs(pr_, "fp32")
        for k, v in over.items():
            setattr(p, k, v)
        return pf.lib().pf_energy_solute_noalloc(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), 0, 0,
                                                 ptr, ptr, ptr, ctypes.c_void_p(out.data_ptr()), None)

    assert c_call(dict(pr, n=(1 << 16, 1 << 15))) == pf.PF_EINVAL
    assert "2^30" in pf.lib().pf_last_error(None).decode()
    bad = dict(pr, lap=19)
    with pytest.raises(pf.PFError, match="lap_stencil"):
        pf.energy_solute_noalloc(bad, t, t, t, out)
    # descriptions pf_create rejects: an unknown interpolation code, a
    # one-sided periodic axis
    assert c_call(pr, interp=7) == pf.PF_EINVAL
    assert "interp" in pf.lib().pf_last_error(None).decode()
    with pytest.raises(pf.PFError, match="periodic"):
        pf.energy_solute_noalloc(dict(pr, bc_lo=("periodic", "noflux")), t, t, t, out)
    # tensors that do not fit the grid or the precision never reach the kernel
    with pytest.raises(pf.PFError, match="elements"):
        pf.energy_solute_noalloc(pr, t, t[:63], t, out)
    with pytest.raises(pf.PFError, match="float64"):
        pf.energy_solute_noalloc(pr, t, t, t, out.float())
    with pytest.raises(pf.PFError, match="float64"):
        pf.energy_solute_noalloc(pr, t, t, t, out[:1])
