"""Parity at the benchmarked configuration (3D sphere seed, 19-point
Laplacian, no-flux box, FP32 step) beyond the short full-size runs:

* the FP64 kernel over the 3000-step sphere that the FP32 test holds at a
  conditioning-limited bar, at the FP64 bar: the FP32 gap is rounding, not a
  kernel error;
* the full 256^3 grid in the launch configuration the benchmark times, with
  A = 1.5 and b = 0.3, so that every (1-A) term (anti-trapping current, cross
  term of the phi equation, K correction) and every b term is live;
* the benchmark's own recipe (undercooling 0.5, k_e = 0.1, D_s/D_l = 1e-4,
  dx = W/2) on a 64^3 box with the seed radius scaled by the box (5 cells) for
  the full 5x10^3 steps, in FP32, at the stated FP32 bars.
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300.pf import Sim

from conftest import rel_err
from test_gpu_parity import TOL64, assert_fields, run_pair, total_c

pytestmark = pytest.mark.gpu


def test_fp64_sphere_3000_steps():
    """The sphere of test_fp32_3d_sphere_3000_steps (70 x 38 x 33, undercooling
    0.2, the solid fraction growing from 8 % to 89 %), in FP64 on the GPU: every
    field at the FP64 bar after the same 3000 steps."""
    pr, phi, cs, cl = wl.sphere_seed_3d(n=(70, 38, 33), radius_cells=12.0, u=0.2, A=1.0, b=1.0)
    phi, cs, cl = (np.asarray(a, np.float32).astype(np.float64) for a in (phi, cs, cl))
    st, g, _ = run_pair(pr, phi, cs, cl, 3000)
    assert_fields(st, g, TOL64, pr)


@pytest.fixture(scope="module")
def sphere256_A15():
    return wl.sphere_seed_3d(n=256, radius_cells=20.0, A=1.5, b=0.3)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sphere_256_cubed_all_terms_live(sphere256_A15, precision):
    """The 256^3 launch (8 x 16 x 7 CTAs, z-chunks of 37 planes) with A = 1.5,
    b = 0.3, two steps, every cell compared: FP64 at the FP64 bar (oracle
    spread measured on one perturbed run), FP32 within 1e-5 in phi and within
    the stated FP32 bar of 1e-5 in the total concentration (measured ~1e-6:
    two steps of FP32 arithmetic and the FP32 read-back)."""
    pr, phi, cs, cl = sphere256_A15
    assert tuple(pr["n"]) == (256, 256, 256) and pr["lap"] == 19 and pr["A"] == 1.5 and pr["b"] == 0.3
    if precision == "fp64":
        st, g, _ = run_pair(pr, phi, cs, cl, 2, "fp64")
        assert_fields(st, g, TOL64, pr, reps=1)
        return
    st, g, _ = run_pair(pr, phi, cs, cl, 2, "fp32")
    g = [a.astype(np.float64) for a in g]
    assert np.abs(g[0] - st.phi).max() <= 1e-5, np.abs(g[0] - st.phi).max()
    _, cg = total_c(pr, *g)
    _, co = total_c(pr, st.phi, st.cs, st.cl)
    assert rel_err(cg, co) <= 1e-5, rel_err(cg, co)


def test_fp32_benchmark_recipe_64_cubed_5000_steps():
    """The benchmark's recipe on a 64^3 box, FP32 kernel against the FP64
    oracle from the same FP32-rounded start, at the stated FP32 bars (phi within
    1e-4, total c within 1e-5 relative, solute drift within 1e-7) at two
    checkpoints: step 1000, while the seed grows through the box (solid fraction
    0.39; in the FP64 oracle a relative change of 1e-6 in theta moves phi by
    4.8e-5 here, in H by 1.7e-5), and step 5000, the full run (the box has
    solidified by step 2000; c_s keeps diffusing).  The phase concentrations are
    compared where they are physical (c_s in the solid, c_l in the liquid)."""
    pr, phi, cs, cl = wl.sphere_seed_3d(n=64, radius_cells=5.0, A=1.0, b=1.0)
    assert pr["theta_ref"] == wl.theta_from_undercooling(0.1, 0.5) and pr["D_s"] == 1e-4 and pr["dx"] == 0.5
    phi, cs, cl = (np.asarray(a, np.float32).astype(np.float64) for a in (phi, cs, cl))
    st = oracle.State(pr, phi, cs, cl)
    with Sim(pr, "fp32") as s:
        s.set_fields(phi, cs, cl)
        S0 = s.solute_total()
        done = 0
        for upto in (1000, 5000):
            st.step(upto - done)
            s.step(upto - done)
            done = upto
            g = [a.astype(np.float64) for a in s.get_fields()]
            dphi = np.abs(g[0] - st.phi).max()
            po, co = total_c(pr, st.phi, st.cs, st.cl)
            _, cg = total_c(pr, *g)
            ec = rel_err(cg, co)
            print(f"step {upto}: phi {dphi:.2e}, total c {ec:.2e}, solid fraction {(po >= 0.5).mean():.3f}")
            assert dphi <= 1e-4, (upto, dphi)
            assert ec <= 1e-5, (upto, ec)
            sol, liq = po >= 0.5, po <= 0.5
            assert np.abs(g[1] - st.cs)[sol].max() <= 1e-4 * np.abs(st.cs[sol]).max()
            if liq.any():
                assert np.abs(g[2] - st.cl)[liq].max() <= 1e-4 * np.abs(st.cl[liq]).max()
        S1 = s.solute_total()
    assert abs(S1 - S0) <= 1e-7 * abs(S0), abs(S1 - S0) / abs(S0)


def test_sphere_256_cubed_energy_and_solute_over_300_steps():
    """Properties that hold at any size, checked at the benchmark's full size
    and launch configuration: the discrete free energy (Eq. model1.1) of the
    isothermal sphere never increases from one step to the next (check (a),
    the variational construction) and the total solute stays put (check (b);
    FP32 state, FP64 sums) over 300 steps, F_h recorded on the device after
    every step."""
    import bench
    pr, phi, cs, cl = bench.workload(256)
    assert pr["G_theta"] == 0.0 and pr["v_pull"] == 0.0
    f32 = [np.asarray(a, np.float32) for a in (phi, cs, cl)]
    with Sim(pr, "fp32") as s:
        s.set_fields(*f32)
        S0 = s.solute_total()
        F = s.step_energies(300)
        S1 = s.solute_total()
    dF = np.diff(F)
    print(f"F_h {F[0]:.9e} -> {F[-1]:.9e}, largest increase {dF.max():.2e}, solute drift {abs(S1 - S0) / S0:.2e}")
    assert np.all(dF <= 1e-12 * abs(F[0])), dF.max()
    assert F[-1] < F[0]
    assert abs(S1 - S0) <= 1e-7 * abs(S0)


def test_planar_1d_fp64_full_configuration():
    """The 1D planar front exactly as configured (N = 1024, dx = W/4, FP64,
    front at cell 256, k_e = 0.1, undercooling 0.3, D_s/D_l = 1e-4, no-flux,
    0.9 of the stable dt, 2x10^4 steps) against the oracle: every field at the
    FP64 bar, F_h recorded after every step on the device never increasing and
    equal to the oracle's at the last step, the front position equal."""
    pr, phi, cs, cl = wl.planar_1d(A=2.0, b=1.0)
    assert pr["n"] == (1024,) and pr["dx"] == 0.25
    st = oracle.State(pr, phi, cs, cl)
    st.step(20000)
    with Sim(pr, "fp64") as s:
        s.set_fields(phi, cs, cl)
        F = s.step_energies(20000)
        g = s.get_fields()
        xf, _, cm = s.front()
    st.inputs = (phi, cs, cl, 20000)
    assert_fields(st, g, TOL64, pr, reps=1)
    assert np.all(np.diff(F) <= 1e-12 * abs(F[0]))
    assert abs(F[-1] - st.energy()) <= 1e-12 * abs(F[-1])
    oxf, ocm = st.front()
    assert abs(xf - oxf) <= 1e-12 * abs(oxf) and abs(cm - ocm) <= 1e-12 * abs(ocm)


def test_perturbed_2d_1024_fp32_energy_and_solute_over_1e4_steps():
    """The 2D perturbed front at its full size (1024^2 FP32, 9-point
    Laplacian, periodic along the front, 10^4 steps) through properties that
    hold at any size: F_h never increases from one step to the next (check
    (a)) and the solute drifts by at most 1e-7 relative (check (b))."""
    pr, phi, cs, cl = wl.perturbed_front_2d(A=1.0, b=1.0)
    assert tuple(pr["n"]) == (1024, 1024) and pr["G_theta"] == 0.0
    with Sim(pr, "fp32") as s:
        s.set_fields(*(np.asarray(a, np.float32) for a in (phi, cs, cl)))
        S0 = s.solute_total()
        F = s.step_energies(10000)
        S1 = s.solute_total()
    dF = np.diff(F)
    print(f"F_h {F[0]:.9e} -> {F[-1]:.9e}, largest increase {dF.max():.2e}, solute drift {abs(S1 - S0) / S0:.2e}")
    assert np.all(dF <= 1e-12 * abs(F[0])), dF.max()
    assert abs(S1 - S0) <= 1e-7 * abs(S0)
