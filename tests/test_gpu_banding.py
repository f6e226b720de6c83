"""The band-forming workload of Sec. "Oscillations and solute bands" (Si-As
at G = 1.4e6 K/m, D_s/D_l = 1e-3, pulled at 0.1-0.5 m/s) through the batched
pulled-front kernel, FP64 against the oracle: every field after 2x10^4 steps
(2000 time units, 360 to 1800 window shifts) at the batch bar."""
import numpy as np
import pytest

import oracle
from paper_2303_09671_gb300 import pf
from paper_2303_09671_gb300 import workloads as wl

from conftest import rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("A,b", [(1.0, 1.0), (1.5, 0.1)])
def test_banding_fronts_fp64_match_oracle(A, b):
    vps = [0.1, 0.3, 0.5]
    n, steps = 4096, 20000
    made = [wl.banding_front(v, A=A, b=b, N=n, front_cell=3000) for v in vps]
    prs = [m[0] for m in made]
    vs = [pr["v_pull"] for pr in prs]
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    phi, cs, cl = (np.concatenate([m[i] for m in made]) for i in (1, 2, 3))
    res = pf.run_batch(prs[0], [n] * len(vs), vs, phi, cs, cl, precision="fp64", dt=dts, max_steps=steps,
                       steps_per_launch=2500, launches_per_graph=4, check_every=steps, tol=-1.0,
                       want_fields=True)
    assert (res["steps"] == steps).all()
    for i, (pr, dt) in enumerate(zip(prs, dts)):
        st = oracle.State(dict(pr, dt=dt), *(a[i * n:(i + 1) * n] for a in (phi, cs, cl)))
        st.step(steps)
        assert st.clock.shifts == int(np.floor(pr["v_pull"] * steps * dt / pr["dx"])) >= 300
        g = [res[k][i * n:(i + 1) * n] for k in ("phi", "cs", "cl")]
        for a, o in zip(g, (st.phi, st.cs, st.cl)):
            assert rel_err(a, o) <= 1e-11, (vps[i], rel_err(a, o))
        _, cm = st.front()
        assert abs(res["k_v"][i] - pr["c_inf"] / cm) <= 1e-11
