"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times: the 3D 256^3 sphere seed (19-point Laplacian, no-flux box)
and the 2D 1024^2 perturbed front (9-point Laplacian, periodic along the
front).  The oracle advances the whole grid a few steps (about ten seconds a
step in 3D), so every cell is compared, not a sample."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300.pf import Sim

from conftest import rel_err

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402  (the benchmark's own workload definition)


@pytest.fixture(scope="module")
def sphere256():
    return bench.workload(256)


def total_c(pr, phi, cs, cl):
    f = phi
    p = f ** 3 * (6 * f * f - 15 * f + 10) + pr["a"] * (f - 0.5) * (f * (1 - f)) ** 2
    return p * cs + (1 - p) * cl


def advance(pr, state, nsteps, precision):
    dt = np.float64 if precision == "fp64" else np.float32
    phi, cs, cl = (np.asarray(a, dtype=dt).astype(np.float64) for a in state)
    st = oracle.State(pr, phi, cs, cl)
    st.step(nsteps)
    with Sim(pr, precision) as s:
        s.set_fields(phi, cs, cl)
        s.step(nsteps)
        g = [a.astype(np.float64) for a in s.get_fields()]
    return st, g


def check(pr, st, g, precision):
    if precision == "fp64":
        for name, a, b in zip(("phi", "cs", "cl"), g, (st.phi, st.cs, st.cl)):
            e = rel_err(a, b)
            assert e <= 1e-12, f"{name}: {e:.2e}"
    else:
        # a few FP32 steps: far inside the 1e-4 / 1e-5 bars that hold after 10^4
        assert np.abs(g[0] - st.phi).max() <= 1e-5, np.abs(g[0] - st.phi).max()
        e = rel_err(total_c(pr, *g), total_c(pr, st.phi, st.cs, st.cl))
        assert e <= 1e-6, f"total c: {e:.2e}"


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sphere_256_cubed(sphere256, precision):
    pr, phi, cs, cl = sphere256
    assert tuple(pr["n"]) == (256, 256, 256) and pr["lap"] == 19
    st, g = advance(pr, (phi, cs, cl), 2, precision)
    check(pr, st, g, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_perturbed_front_1024_squared(precision):
    pr, phi, cs, cl = wl.perturbed_front_2d(A=1.0, b=1.0)
    assert tuple(pr["n"]) == (1024, 1024) and pr["lap"] == 9
    st, g = advance(pr, (phi, cs, cl), 50, precision)
    check(pr, st, g, precision)
