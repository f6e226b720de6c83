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


def test_sphere_256_cubed_overlapped_upload(sphere256):
    """The end-to-end path the benchmark times: pf_set_fields_step from
    page-locked host memory (16-plane slabs converted while the first step's
    chunks run) leaves the 256^3 state bit for bit equal to pf_set_fields then
    pf_step, which the test above holds to the oracle."""
    torch = pytest.importorskip("torch")
    pr, phi, cs, cl = sphere256
    f32 = [np.ascontiguousarray(a, dtype=np.float32) for a in (phi, cs, cl)]
    pinned = [torch.from_numpy(a).pin_memory() for a in f32]
    with Sim(pr, "fp32") as s:
        s.set_fields(*f32)
        s.step(2)
        want = s.get_fields()
    with Sim(pr, "fp32") as s:
        s.set_fields_step(*[p.numpy() for p in pinned], n=2)
        got = s.get_fields()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_perturbed_front_1024_squared(precision):
    pr, phi, cs, cl = wl.perturbed_front_2d(A=1.0, b=1.0)
    assert tuple(pr["n"]) == (1024, 1024) and pr["lap"] == 9
    st, g = advance(pr, (phi, cs, cl), 50, precision)
    check(pr, st, g, precision)


def test_beyond_2_31_cells_planar_3d():
    """A 3D FP32 grid of 2048 x 1024 x 1040 = 2.18e9 cells (more than 2^31) with a
    planar front along x, set and read through device pointers: after three
    steps every (y, z) column is the same, bit for bit (64-bit cell indexing
    everywhere), and a column follows the FP64 oracle's 1D run to 1e-5."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = 2048, 1024, 1040
    cells = nx * ny * nz
    assert cells > 2 ** 31
    # the handle's 8 state arrays and the 6 field tensors, 4 B each
    if torch.cuda.mem_get_info()[0] < 1.1 * 14 * 4 * cells:
        pytest.skip("not enough device memory for a grid beyond 2^31 cells")
    pr1, phi1, cs1, cl1 = wl.planar_1d(N=nx, dx=0.5, front_cell=nx // 2, A=1.0, b=1.0)
    pr3 = dict(pr1, dim=3, n=(nx, ny, nz), lap=19, bc_lo=("noflux", "periodic", "periodic"),
               bc_hi=("noflux", "periodic", "periodic"))
    pr3["dt"] = 0.9 * wl.stable_dt(pr3)
    pr1 = dict(pr1, dt=pr3["dt"])
    f1 = [np.asarray(a, np.float32) for a in (phi1, cs1, cl1)]
    st = oracle.State(pr1, *(a.astype(np.float64) for a in f1))
    st.step(3)
    dev = [torch.from_numpy(a).cuda().reshape(1, 1, nx).expand(nz, ny, nx).contiguous() for a in f1]
    with Sim(pr3, "fp32") as s:
        s.set_fields(*dev)
        del dev
        s.step(3)
        out = [torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
        s.get_fields(out=out)
    for a in out:
        col = a[:1, :1, :]
        assert bool(torch.eq(a, col).all()), "columns differ"
    got = out[0][0, 0].double().cpu().numpy()
    assert np.abs(got - st.phi).max() <= 1e-5, np.abs(got - st.phi).max()
