"""Failure detection on the host: a non-finite value planted in the input
propagates through the step (harmlessly for the GPU) and the FP64 diagnostics
report PF_ENONFINITE; the handle stays usable afterwards."""
import numpy as np
import pytest

from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300.pf import PFError, Sim

pytestmark = pytest.mark.gpu

PF_ENONFINITE = -4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_non_finite_state_is_reported_and_recoverable(precision):
    pr, phi, cs, cl = wl.random_state(3, (37, 19, 13), dx=0.5, A=1.5, b=0.3, seed=3)
    bad = cl.copy()
    bad.flat[bad.size // 2] = np.nan
    with Sim(pr, precision) as s:
        s.set_fields(phi, cs, bad)
        s.step(3)
        for call in (s.energy, s.solute_total):
            with pytest.raises(PFError) as e:
                call()
            assert e.value.code == PF_ENONFINITE
        s.set_fields(phi, cs, cl)
        s.step(3)
        assert np.isfinite(s.energy()) and np.isfinite(s.solute_total())


def test_allocation_failure_is_reported_and_recoverable():
    """A grid whose state does not fit in device memory (2^34 cells in FP64,
    eight arrays of 137 GB) fails in pf_create with PF_ENOMEM, frees what it
    had allocated, and the next handle works.  The failing call is the real
    cudaMalloc; nothing is launched."""
    from paper_2303_09671_gb300 import pf
    pr, phi, cs, cl = wl.random_state(3, (16, 8, 8), dx=0.5, A=1.5, b=0.3, seed=4)
    big = dict(pr, n=(1024, 1024, 16384))
    with pytest.raises(PFError) as e:
        Sim(big, "fp64")
    assert e.value.code == pf.PF_ENOMEM
    with Sim(pr, "fp64") as s:
        s.set_fields(phi, cs, cl)
        s.step(2)
        assert np.isfinite(s.energy())
