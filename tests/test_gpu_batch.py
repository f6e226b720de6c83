"""Batched 1D pulled fronts (pf_run_batch) against the FP64 oracle and the
single-instance path."""
import numpy as np
import pytest

import oracle
from paper_2303_09671_gb300 import workloads as wl
from paper_2303_09671_gb300 import pf

from conftest import rel_err

pytestmark = pytest.mark.gpu


def batch_inputs(lengths, vs, A=1.0, b=1.0, dx=0.5, front_cell=24):
    """Instances share the frozen temperature (x0 = front_cell dx, theta_ref)."""
    prs, phis, css, cls = [], [], [], []
    for n, v in zip(lengths, vs):
        pr, phi, cs, cl = wl.pulled_front_1d(N=n, dx=dx, V=v, A=A, b=b, front_cell=front_cell)
        prs.append(pr)
        phis.append(phi)
        css.append(cs)
        cls.append(cl)
    return prs, np.concatenate(phis), np.concatenate(css), np.concatenate(cls)


def oracle_runs(prs, lengths, phis, css, cls, dts, nsteps):
    out, o = [], 0
    for pr, n, dt in zip(prs, lengths, dts):
        st = oracle.State(dict(pr, dt=dt), phis[o:o + n], css[o:o + n], cls[o:o + n])
        st.step(nsteps)
        out.append(st)
        o += n
    return out


def test_batch_fp64_matches_oracle():
    """Four instances of different lengths and velocities, 300 steps (3 graph
    replays of 2 launches x 50 steps) with window shifts."""
    lengths = [64, 200, 333, 512]
    vs = [0.05, 0.1, 0.2, 0.3]
    prs, phi, cs, cl = batch_inputs(lengths, vs)
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    res = pf.run_batch(prs[0], lengths, vs, phi, cs, cl, precision="fp64", dt=dts, max_steps=300,
                       steps_per_launch=50, launches_per_graph=2, check_every=100, tol=-1.0,
                       want_fields=True)
    assert (res["steps"] == 300).all() and not res["converged"].any()
    ref = oracle_runs(prs, lengths, phi, cs, cl, dts, 300)
    o = 0
    for n, st in zip(lengths, ref):
        assert st.clock.shifts > 0
        for a, b_ in ((res["phi"][o:o + n], st.phi), (res["cs"][o:o + n], st.cs), (res["cl"][o:o + n], st.cl)):
            assert rel_err(a, b_) <= 1e-11, rel_err(a, b_)
        o += n


@pytest.mark.parametrize("cpt", [1, 2, 8])
def test_batch_fp32_matches_single_instance_path(cpt):
    lengths = [96, 300, 700]
    vs = [0.1, 0.2, 0.4]
    prs, phi, cs, cl = batch_inputs(lengths, vs)
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    res = pf.run_batch(prs[0], lengths, vs, phi, cs, cl, precision="fp32", dt=dts, max_steps=400,
                       steps_per_launch=100, launches_per_graph=2, check_every=100, tol=-1.0,
                       want_fields=True, cells_per_thread=cpt)
    o = 0
    for pr, n, dt in zip(prs, lengths, dts):
        with pf.Sim(dict(pr, dt=dt), "fp32") as s:
            s.set_fields(phi[o:o + n], cs[o:o + n], cl[o:o + n])
            s.step(400)
            g = s.get_fields()
        assert np.abs(res["phi"][o:o + n] - g[0]).max() <= 1e-5
        assert rel_err(res["cs"][o:o + n], g[1]) <= 1e-5 and rel_err(res["cl"][o:o + n], g[2]) <= 1e-5
        o += n


def test_batch_autotunes_and_converges():
    """A small sweep run until each instance reaches a steady k_v (after the
    temperature has been pulled 200 W): all converge, 0 < k_v <= 1."""
    lengths = [512, 1024, 768]
    vs = [2.0, 0.5, 1.0]
    prs, phi, cs, cl = batch_inputs(lengths, vs, front_cell=128)
    res = pf.run_batch(prs[0], lengths, vs, phi, cs, cl, precision="fp32", max_steps=400000,
                       steps_per_launch=1000, launches_per_graph=4, check_every=200, window=2.0,
                       tol=1e-6, min_travel=200.0)
    assert res["cells_per_thread"] in (1, 2, 4, 8)
    assert res["converged"].all(), res
    assert ((res["k_v"] > 0) & (res["k_v"] <= 1 + 1e-6)).all(), res["k_v"]
    assert (res["t"] * np.asarray(vs) >= 200.0).all()


def test_batch_rejects_invalid():
    prs, phi, cs, cl = batch_inputs([64], [0.1])
    with pytest.raises(pf.PFError):
        pf.run_batch(prs[0], [4], [0.1], phi[:4], cs[:4], cl[:4])
    with pytest.raises(pf.PFError):
        pf.run_batch(prs[0], [64], [-1.0], phi, cs, cl)


def test_closed_box_planar_front_with_energy_records():
    """The 1D planar front (N = 1024, dx = W/4, FP64, no-flux at both ends) as
    one persistent instance recording F_h after every step: fields and F_h
    against the oracle, and F_h non-increasing (check (a))."""
    pr, phi, cs, cl = wl.planar_1d(A=2.0, b=1.0)
    n, steps = pr["n"][0], 2000
    res = pf.run_batch(pr, [n], [0.0], phi, cs, cl, precision="fp64", dt=[pr["dt"]], max_steps=steps,
                       steps_per_launch=500, launches_per_graph=2, check_every=steps, tol=-1.0,
                       want_fields=True, energy_every=1)
    st = oracle.State(pr, phi, cs, cl)
    hist = st.step(steps + 1, energy=True)      # hist[s] = F_h before step s
    ref = oracle.State(pr, phi, cs, cl)
    ref.step(steps)
    for a, b_ in ((res["phi"], ref.phi), (res["cs"], ref.cs), (res["cl"], ref.cl)):
        assert rel_err(a, b_) <= 1e-11, rel_err(a, b_)
    E = res["energy"][0]
    assert np.all(np.isfinite(E))
    assert np.abs(E - hist[1:steps + 1]).max() <= 1e-12 * np.abs(hist).max()
    assert np.all(np.diff(E) <= 1e-13 * abs(E[0]))


def test_batch_stops_exactly_at_max_steps():
    """A step cap that is not a multiple of the graph replay (4 launches of 100
    steps): three replays and a directly launched remainder of 34 steps, and the
    fields equal those of one 1234-step launch bit for bit."""
    lengths, vs = [96, 300], [0.1, 0.2]
    prs, phi, cs, cl = batch_inputs(lengths, vs)
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    common = dict(precision="fp64", dt=dts, check_every=50, tol=-1.0, want_fields=True, cells_per_thread=2)
    a = pf.run_batch(prs[0], lengths, vs, phi, cs, cl, max_steps=1234, steps_per_launch=100,
                     launches_per_graph=4, **common)
    b = pf.run_batch(prs[0], lengths, vs, phi, cs, cl, max_steps=1234, steps_per_launch=1234,
                     launches_per_graph=1, **common)
    assert (a["steps"] == 1234).all() and (b["steps"] == 1234).all()
    for k in ("phi", "cs", "cl"):
        assert np.array_equal(a[k], b[k]), k
