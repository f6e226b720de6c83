"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test checks the oracle against something other than itself:
closed forms printed in the paper, a continuum model derived symbolically from
the free-energy functional, exact invariants, special cases that reduce to
textbook results, and convergence orders.  Planted mistakes (oracle PLANT
bits) show that the pins catch a dropped term, a wrong sign or a swapped
operand.
"""
import math

import numpy as np
import pytest
import sympy as sp
from scipy.linalg import solve_banded

import oracle
from paper_2303_09671_gb300 import workloads as wl

import bruteforce
from continuum import ContinuumModel, X, Y
from conftest import rel_err

I_DW = 1.0 / (3.0 * math.sqrt(2.0))


def base(dim=1, n=(64,), k_e=0.1, theta=2.0, D_s=0.1, **kw):
    kw.setdefault("dt", 1e-3)
    return wl.scaled_params(dim, n, 0.5, k_e, theta, D_s, **kw)


# ------------------------------------------------------------- pointwise pins

@pytest.mark.parametrize("k_e,theta", [(0.1, 3.7), (0.3, 1.0), (0.15, 2.7), (0.5, 1.3)])
@pytest.mark.parametrize("phi", [0.0, 0.3, 0.5, 0.9])
@pytest.mark.parametrize("A", [0.0, 0.4, 2.0])
def test_equilibrium_pair_has_zero_driving_force(k_e, theta, phi, A):
    """At (c_s, c_l) = (k_e theta, theta): mu_s = mu_l (Eq. dil2) and the driving
    force vanishes (common tangent, Eq. dil5.1), for any phi and A."""
    pr = base(k_e=k_e, A=A, b=0.3, a=0.2)
    pr["theta_ref"] = theta
    q = oracle.point(pr, phi, k_e * theta, theta, theta)
    assert abs(q["mu_s"] - q["mu_l"]) <= 1e-14
    assert abs(q["dG"]) <= 1e-13


@pytest.mark.parametrize("cs,cl,theta", [(0.07, 1.3, 2.0), (0.4, 0.9, 3.7), (1.0, 1.9, 10.0)])
def test_driving_forces_match_closed_forms(cs, cl, theta):
    """f_s - f_l - (c_s - c_l) mu_s and f_s - f_l - (c_s - c_l) mu_l against the
    closed forms of Eqs. dil5.1 / dil5.2 (scaled units, c_l^eq = theta)."""
    k = 0.1
    pr = base(k_e=k)
    q = oracle.point(pr, 0.5, cs, cl, theta)
    d = cs - cl
    g_s = q["f_s"] - q["f_l"] - d * q["mu_s"]
    g_l = q["f_s"] - q["f_l"] - d * q["mu_l"]
    assert abs(g_s - (cl * math.log(cs / (k * cl)) + theta * (k - 1) - d)) <= 1e-13
    assert abs(g_l - (cs * math.log(cs / (k * cl)) + theta * (k - 1) - d)) <= 1e-13


@pytest.mark.parametrize("interp", ["quintic", "cubic"])
@pytest.mark.parametrize("a", [0.0, 0.7, -1.3])
def test_interpolation_constraints(interp, a):
    """p(0) = 0, p(1) = 1, p'(0) = p'(1) = 0 (text after Eq. interpolation2),
    p(1-phi) = 1 - p(phi) (antisymmetry), and p' is the derivative of p."""
    pr = base(interp=interp, a=a)
    P = lambda f: oracle.point(pr, f, 1.0, 1.0, 1.0)
    assert P(0.0)["p"] == 0.0 and abs(P(1.0)["p"] - 1.0) <= 1e-15
    assert P(0.0)["dp"] == 0.0 and abs(P(1.0)["dp"]) <= 1e-15
    for f in np.linspace(0.05, 0.95, 7):
        assert abs(P(1 - f)["p"] - (1 - P(f)["p"])) <= 1e-14
        h = 1e-6
        fd = (P(f + h)["p"] - P(f - h)["p"]) / (2 * h)
        assert abs(fd - P(f)["dp"]) <= 1e-8


def test_quintic_h_is_the_paper_polynomial():
    pr = base(a=0.0)
    for f in np.linspace(0, 1, 11):
        assert abs(oracle.point(pr, f, 1, 1, 1)["p"] - f ** 3 * (6 * f * f - 15 * f + 10)) <= 1e-15


@pytest.mark.parametrize("cs,cl", [(0.1, 1.0), (0.3, 2.0)])
def test_choice_one_reduction(cs, cl):
    """b = 1, a = 0 recovers the first choice of Sec. "Choice of interpolation
    functions": h_n = h, 1/q_n = h/M_s + (1-h)/M_l (Eq. inverse) and the
    anti-trapping function of Eq. antitrapping2."""
    pr = base(b=1.0, a=0.0, D_s=1e-3)
    for f in (0.1, 0.5, 0.8):
        q = oracle.point(pr, f, cs, cl, 1.0)
        h = f ** 3 * (6 * f * f - 15 * f + 10)
        Ms, Ml = pr["D_s"] * cs, pr["D_l"] * cl
        assert abs(q["h_n"] - h) <= 1e-15
        assert abs(1 / q["q_n"] - (h / Ms + (1 - h) / Ml)) <= 1e-10 * (1 / q["q_n"])
        at2 = (Ms - Ml) * h * (1 - h) / (Ms * (1 - h) + Ml * h)
        assert abs(q["a_phi"] - at2) <= 1e-14


def test_qn_limits_and_normal_interpolation():
    """q_n(p=0) = M_l, q_n(p=1) = M_s; 1/q_n = h_n/M_s + (1-h_n)/M_l (Eq. normal2)."""
    pr = base(b=0.02, a=0.3, D_s=1e-3)
    cs, cl = 0.2, 1.4
    Ms, Ml = pr["D_s"] * cs, pr["D_l"] * cl
    assert abs(oracle.point(pr, 0.0, cs, cl, 1)["q_n"] - Ml) <= 1e-15
    assert abs(oracle.point(pr, 1.0, cs, cl, 1)["q_n"] - Ms) <= 1e-15
    for f in (0.2, 0.5, 0.7):
        q = oracle.point(pr, f, cs, cl, 1)
        assert abs(1 / q["q_n"] - (q["h_n"] / Ms + (1 - q["h_n"]) / Ml)) <= 1e-12 / q["q_n"]
        # anti-trapping function of Eq. shape_function = w_s p - w_l (1 - p) (Eq. antitrapping)
        assert abs(q["a_phi"] - (q["w_s"] * q["p"] - q["w_l"] * (1 - q["p"]))) <= 1e-15


def test_drag_coefficient_limits():
    """The re-derived drag: D = M_s^n/(M_s^n + M_l^n) at A = 0 and D = p at A = 1
    (the KKS-like limit, Sec. "KKS"), linear in A, inside [0, 1] for A in [0, 1]."""
    for f in (0.1, 0.5, 0.9):
        q0 = oracle.point(base(A=0.0, b=0.3), f, 0.2, 1.1, 1)
        q1 = oracle.point(base(A=1.0, b=0.3), f, 0.2, 1.1, 1)
        qh = oracle.point(base(A=0.5, b=0.3), f, 0.2, 1.1, 1)
        assert abs(q0["drag"] - q0["w_s"]) <= 1e-15
        assert abs(q1["drag"] - q1["p"]) <= 1e-15
        assert abs(qh["drag"] - 0.5 * (q0["drag"] + q1["drag"])) <= 1e-15
        assert 0.0 <= qh["drag"] <= 1.0


# ------------------------------------------------- continuum-model convergence

LX = 8.0
PHI_E = 1 / (1 + sp.exp(sp.sqrt(2) * (X - 4 - 0.6 * sp.sin(2 * sp.pi * Y / LX))))
CS_E = 0.12 * (1 + 0.3 * sp.sin(2 * sp.pi * X / LX) * sp.cos(2 * sp.pi * Y / LX)
               + 0.1 * sp.cos(2 * sp.pi * Y / LX))
CL_E = 1.1 + 0.25 * sp.cos(2 * sp.pi * X / LX + 0.3) * sp.sin(2 * sp.pi * Y / LX + 0.5)
PHI_1D = 1 / (1 + sp.exp(sp.sqrt(2) * (X - 4)))
CS_1D = 0.12 * (1 + 0.3 * sp.sin(2 * sp.pi * X / LX))
CL_1D = 1.1 + 0.25 * sp.cos(2 * sp.pi * X / LX + 0.3)


def continuum_errors(dim, ns, plant=0, **kw):
    errs = []
    for n in ns:
        dx = LX / n
        if dim == 2:
            pr = wl.scaled_params(2, (n, n), dx, 0.1, 2.0, 0.1, delta=1e-9, dt=1e-3,
                                  bc_lo=("noflux", "periodic"), bc_hi=("noflux", "periodic"), **kw)
            fields = (PHI_E, CS_E, CL_E)
        else:
            pr = wl.scaled_params(1, (n,), dx, 0.1, 2.0, 0.1, delta=1e-9, dt=1e-3, **kw)
            fields = (PHI_1D, CS_1D, CL_1D)
        pr["plant"] = plant
        cm = ContinuumModel(pr, *fields)
        xc = (np.arange(n) + 0.5) * dx
        if dim == 2:
            Xg, Yg = np.meshgrid(xc, xc, indexing="xy")
        else:
            Xg, Yg = xc, np.zeros_like(xc)
        vals = [sp.lambdify((X, Y), e)(Xg, Yg) * np.ones_like(Xg) for e in fields]
        st = oracle.State(pr, *vals)
        r_or = st.rates()
        r_co = cm.rates(Xg, Yg)
        m = 3 * (n // 16)
        sl = (slice(None), slice(m, n - m)) if dim == 2 else slice(m, n - m)
        errs.append([np.abs(a[sl] - b[sl]).max() / np.abs(b[sl]).max() for a, b in zip(r_or, r_co)])
    return np.array(errs)


@pytest.mark.parametrize("A", [0.0, 0.4, 1.0, 2.0])
def test_rates_converge_to_functional_model_2d(A):
    """phidot, dc/dt and dd/dt of the oracle converge at second order (Sec.
    "Numerical technique") to the rates of the general model built from the
    functional, Eqs. model10-model14, model7-model8 with the interpolation choices
    of Sec. "Alternative choice of interpolation functions".  This pins the
    re-derived driving force, the anti-trapping and cross terms, and the
    normal/tangential split."""
    e = continuum_errors(2, (16, 32, 64), A=A, b=0.3, a=0.2, G_theta=0.05, v_pull=0.1, x0=2.0)
    ratio = e[:-1] / e[1:]
    assert (ratio[-1] > 3.4).all(), f"convergence ratios {ratio}"
    assert (e[-1] < 0.03).all(), f"errors {e[-1]}"


@pytest.mark.parametrize("opts", [dict(interp="cubic"), dict(mobility="const"), dict(b=1.0, a=0.0)])
def test_rates_converge_to_functional_model_1d(opts):
    e = continuum_errors(1, (16, 32, 64), A=0.4, **{**dict(b=0.3, a=0.2), **opts})
    ratio = e[:-1] / e[1:]
    assert (ratio[-1] > 3.4).all(), f"convergence ratios {ratio}"


@pytest.mark.parametrize("plant", sorted(oracle.PLANT))
def test_planted_mistakes_break_the_continuum_pin(plant):
    """Each planted mistake (the drag as printed in Eq. drivingforce_nonvar, a
    dropped anti-trapping, cross or rate-coefficient term, a wrong projection
    sign, swapped anti-trapping weights, the crystallisation force with mu_s)
    leaves an O(1) error that does not converge."""
    e = continuum_errors(2, (32, 64), plant=oracle.PLANT[plant], A=0.4, b=0.3, a=0.2)
    ratio = e[0] / e[1]
    assert (e[1] > 0.05).any() and (ratio < 2.0).any(), f"{plant}: errors {e[1]}, ratios {ratio}"


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("maker,nsteps", [
    (lambda: wl.planar_1d(N=256, front_cell=64, A=2.0, b=1.0), 3000),
    (lambda: wl.random_state(2, (48, 24), A=1.5, b=0.3, bc_lo=("noflux", "periodic"),
                             bc_hi=("noflux", "periodic")), 300),
    (lambda: wl.random_state(3, (24, 12, 10), A=1.0, b=0.3, lap=19), 100),
    (lambda: wl.random_state(3, (37, 19, 13), A=1.5, b=0.3, lap=7, seed=7,
                             bc_lo=("noflux", "periodic", "periodic"),
                             bc_hi=("noflux", "periodic", "periodic")), 60),
])
def test_total_solute_conserved(maker, nsteps):
    """Check (b): dc/dt = -div J (Eq. model5) telescopes under no-flux and
    periodic boundaries, so S_h is constant up to rounding."""
    pr, phi, cs, cl = maker()
    st = oracle.State(pr, phi, cs, cl)
    S0 = st.solute()
    st.step(nsteps)
    assert abs(st.solute() - S0) <= 2e-13 * abs(S0)


def test_mixture_is_the_pointwise_p_and_the_solute_density():
    """oracle.mixture (the per-cell helper the full-size GPU tests use) gives
    the p(phi) of the pointwise evaluator at every cell, including the pure
    phases (p(0) = 0, p(1) = 1), and c = p c_s + (1 - p) c_l summed times
    dx^dim is the oracle's S_h."""
    for interp in ("quintic", "cubic"):
        pr, phi, cs, cl = wl.random_state(2, (30, 11), A=1.5, b=0.3, a=-0.3, seed=3, interp=interp)
        phi = phi.copy()
        phi[0, 0], phi[0, 1] = 0.0, 1.0
        p, c = oracle.mixture(pr, phi, cs, cl)
        ref = np.array([oracle.point(pr, f, 1.0, 1.0, 0.0)["p"] for f in phi.ravel()]).reshape(phi.shape)
        assert np.array_equal(p, ref)
        assert p[0, 0] == 0.0 and p[0, 1] == 1.0
        assert np.allclose(c, ref * cs + (1 - ref) * cl, rtol=1e-15, atol=0)
        S = oracle.State(pr, phi, cs, cl).solute()
        assert abs(c.sum() * pr["dx"] ** 2 - S) <= 1e-13 * abs(S)


@pytest.mark.parametrize("maker,nsteps", [
    (lambda: wl.planar_1d(N=512, A=2.0, b=1.0), 4000),
    (lambda: wl.perturbed_front_2d(nx=128, ny=128, front=40, seed=20, A=1.5, b=0.3), 1500),
    (lambda: wl.random_state(3, (24, 16, 12), A=1.0, b=0.3), 200),
])
def test_free_energy_never_increases(maker, nsteps):
    """Check (a): the variational construction gives dF/dt <= 0 for positive
    mobilities (text after Eq. model12); the discrete energy decreases every step."""
    pr, phi, cs, cl = maker()
    st = oracle.State(pr, phi, cs, cl)
    E = st.step(nsteps, energy=True)
    assert (np.diff(E) <= 1e-12 * np.abs(E[:-1])).all(), f"max increase {np.diff(E).max():.3e}"
    assert E[-1] < E[0]


# ------------------------------------------------ equilibrium: profile, gamma

def discrete_equilibrium_1d(N, dx, H, sigma):
    """Newton solve of sigma L_h phi = H f_dw'(phi) (3-point, no-flux, N even) in
    the antisymmetric class phi_{N-1-i} = 1 - phi_i, which removes the
    translation mode: only the left half is solved, its right neighbour being
    the mirror image 1 - phi_{N/2-1}."""
    M = N // 2
    x = (np.arange(N) + 0.5) * dx
    u = wl.tanh_profile(x[:M], 0.5 * N * dx)
    c = sigma / dx ** 2
    for _ in range(60):
        left = np.concatenate([u[:1], u[:-1]])                 # mirror ghost at the wall
        right = np.concatenate([u[1:], 1.0 - u[-1:]])          # antisymmetric partner
        Fv = c * (left - 2 * u + right) - H * 2 * u * (1 - u) * (1 - 2 * u)
        diag = -2 * c - H * (2 - 12 * u + 12 * u ** 2)
        diag[0] += c
        diag[-1] -= c
        ab = np.zeros((3, M))
        ab[0, 1:] = c
        ab[1] = diag
        ab[2, :-1] = c
        du = solve_banded((1, 1), ab, -Fv)
        u = u + du
        if np.abs(du).max() < 1e-16:
            break
    return x, np.concatenate([u, 1.0 - u[::-1]])


@pytest.mark.parametrize("A,b,a", [(0.4, 0.3, 0.0), (2.0, 1.0, -0.3), (1.0, 0.05, 0.0)])
def test_flat_front_at_equilibrium_is_a_fixed_point(A, b, a):
    """Check (c): the discrete equilibrium profile with c_s = k_e theta, c_l = theta
    (supplement Eqs. eq4-eq14, Eq. dil2) is stationary: partition k = k_e."""
    theta, k = 2.5, 0.1
    pr = wl.scaled_params(1, (256,), 0.25, k, theta, 1e-3, A=A, b=b, a=a)
    x, phi = discrete_equilibrium_1d(256, 0.25, pr["H"], pr["sigma"])
    cs, cl = np.full(256, k * theta), np.full(256, theta)
    st = oracle.State(pr, phi, cs, cl)
    pd, cd, dd = st.rates()
    assert np.abs(pd).max() <= 1e-12
    st.step(10000)
    assert np.abs(st.phi - phi).max() <= 1e-10
    assert np.abs(st.cs - cs).max() <= 1e-10 and np.abs(st.cl - cl).max() <= 1e-10


def test_equilibrium_profile_and_interface_energy_converge():
    """The discrete equilibrium tends to phi_0 = (1 - tanh(x/(sqrt 2 W)))/2
    (supplement Eq. eq18) and its excess free energy to gamma = I W H with
    I = 1/(3 sqrt 2) (supplement Eq. eq34), both at O(dx^2)."""
    theta, k = 2.0, 0.1
    L = 32.0
    e_prof, e_gam = [], []
    for dx in (0.5, 0.25, 0.125):
        N = int(round(L / dx))
        pr = wl.scaled_params(1, (N,), dx, k, theta, 1e-3, A=1.0, b=1.0)
        x, phi = discrete_equilibrium_1d(N, dx, pr["H"], pr["sigma"])
        exact = 0.5 * (1 - np.tanh((x - L / 2) / math.sqrt(2)))
        e_prof.append(np.abs(phi - exact).max())
        st = oracle.State(pr, phi, np.full(N, k * theta), np.full(N, theta))
        mu_eq, omega = math.log(theta), -theta      # grand potential omega_s = omega_l = -theta
        excess = st.energy() - mu_eq * st.solute() - omega * N * dx
        e_gam.append(abs(excess - I_DW * pr["H"]))
    r_prof = e_prof[0] / e_prof[1], e_prof[1] / e_prof[2]
    r_gam = e_gam[0] / e_gam[1], e_gam[1] / e_gam[2]
    assert all(3.5 < r < 4.5 for r in r_prof), (e_prof, r_prof)
    assert all(3.5 < r < 4.5 for r in r_gam), (e_gam, r_gam)
    assert e_gam[-1] < 1e-3 * I_DW * 10


# ------------------------------------------------ linear modes (closed forms)

@pytest.mark.parametrize("dim,lap,kvec", [
    (1, 3, (3,)), (2, 5, (2, 1)), (2, 9, (2, 2)), (2, 9, (3, 0)), (3, 7, (1, 2, 1)), (3, 19, (2, 1, 1)),
    (3, 19, (0, 2, 2)),
])
def test_allen_cahn_mode_decays_at_the_discrete_rate(dim, lap, kvec):
    """Around the liquid (phi ~ eps cos(k.x)), with the phases at equilibrium,
    phidot = -M_phi (2 H + sigma lam_k) phi + O(eps^2): lam_k is the symbol of
    the Laplacian stencil (weights w_o: lam_k = sum_o w_o (1 - cos(k.o dx)))."""
    n = (16, 16, 16)[:dim]
    pr = wl.scaled_params(dim, n, 0.5, 0.1, 2.0, 0.1, lap=lap, A=0.4, b=0.3, dt=1e-3,
                          bc_lo=("periodic",) * dim, bc_hi=("periodic",) * dim)
    k = [2 * math.pi * kv / (nn * 0.5) for kv, nn in zip(kvec, n)]
    grids = np.meshgrid(*[(np.arange(nn) + 0.5) * 0.5 for nn in n], indexing="ij")
    arg = sum(kk * g for kk, g in zip(k, grids))
    eps = 1e-7
    phi = (eps * np.cos(arg)).transpose()
    theta = pr["theta_ref"]
    st = oracle.State(pr, phi, np.full(phi.shape, 0.1 * theta), np.full(phi.shape, theta))
    pd = st.rates()[0]
    dx = 0.5
    # stencil symbol
    offs = []
    if lap in (3, 5, 7):
        for a in range(dim):
            for s in (-1, 1):
                o = [0] * 3; o[a] = s; offs.append((tuple(o), 1.0))
    elif lap == 9:
        for dy in (-1, 0, 1):
            for dxo in (-1, 0, 1):
                if dxo or dy:
                    offs.append(((dxo, dy, 0), 1 / 6 if (dxo and dy) else 2 / 3))
    else:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dxo in (-1, 0, 1):
                    nz = (dxo != 0) + (dy != 0) + (dz != 0)
                    if nz in (1, 2):
                        offs.append(((dxo, dy, dz), 1 / 3 if nz == 1 else 1 / 6))
    kk = list(k) + [0.0] * (3 - dim)
    lam = sum(w * (1 - math.cos(sum(kk[a] * o[a] * dx for a in range(3)))) for o, w in offs) * 2 / dx ** 2 / 2
    expect = -pr["M_phi"] * (2 * pr["H"] + pr["sigma"] * lam) * phi
    assert np.abs(pd - expect).max() <= 1e-4 * np.abs(expect).max()


def test_liquid_diffusion_mode_decays_at_the_discrete_rate():
    """In the bulk liquid (phi = 0), c_l = theta (1 + eps cos kx) diffuses with
    D_l: dc/dt = -D_l (2 - 2 cos k dx)/dx^2 (c - theta) + O(eps^2)."""
    n, dx = 32, 0.5
    pr = wl.scaled_params(1, (n,), dx, 0.1, 2.0, 0.1, A=0.4, b=0.3, dt=1e-3,
                          bc_lo=("periodic",), bc_hi=("periodic",))
    k = 2 * math.pi * 3 / (n * dx)
    x = (np.arange(n) + 0.5) * dx
    eps = 1e-6
    cl = 2.0 * (1 + eps * np.cos(k * x))
    st = oracle.State(pr, np.zeros(n), np.full(n, 0.2), cl)
    cdot = st.rates()[1]
    lam = (2 - 2 * math.cos(k * dx)) / dx ** 2
    expect = -pr["D_l"] * lam * (cl - 2.0)
    assert np.abs(cdot - expect).max() <= 1e-5 * np.abs(expect).max()


# ------------------------------------------------------------- symmetries

def test_planar_2d_and_3d_equal_1d():
    pr1, phi, cs, cl = wl.random_state(1, (40,), A=1.5, b=0.3, seed=3)
    s1 = oracle.State(pr1, phi, cs, cl)
    s1.step(30)
    for dim, lap, shape in ((2, 9, (5, 40)), (2, 5, (5, 40)), (3, 19, (3, 4, 40)), (3, 7, (3, 4, 40))):
        pr = dict(pr1, dim=dim, lap=lap, n=(40,) + shape[:-1][::-1],
                  bc_lo=("noflux",) + ("periodic",) * (dim - 1), bc_hi=("noflux",) + ("periodic",) * (dim - 1))
        b = lambda a: np.broadcast_to(a, shape).copy()
        s = oracle.State(pr, b(phi), b(cs), b(cl))
        s.step(30)
        for u, v in ((s.phi, s1.phi), (s.cs, s1.cs), (s.cl, s1.cl)):
            assert np.abs(u - v).max() <= 1e-13


def test_z_invariant_3d_19pt_equals_2d_9pt():
    pr2, phi, cs, cl = wl.random_state(2, (30, 16), A=1.5, b=0.3, seed=4)
    s2 = oracle.State(pr2, phi, cs, cl)
    s2.step(20)
    pr3 = dict(pr2, dim=3, lap=19, n=(30, 16, 4), bc_lo=pr2["bc_lo"] + ("periodic",),
               bc_hi=pr2["bc_hi"] + ("periodic",))
    r = lambda a: np.repeat(a[None], 4, axis=0)
    s3 = oracle.State(pr3, r(phi), r(cs), r(cl))
    s3.step(20)
    for u, v in ((s3.phi, s2.phi), (s3.cs, s2.cs), (s3.cl, s2.cl)):
        assert np.abs(u - v[None]).max() <= 1e-13


def test_axis_permutation_equivariance():
    """Without a temperature gradient the step has no preferred axis: the run
    on a transposed state is the transposed run."""
    pr, phi, cs, cl = wl.random_state(2, (20, 28), A=1.5, b=0.3, seed=9)
    pr = dict(pr, bc_lo=("noflux", "dirichlet"), bc_hi=("periodic", "periodic"))
    pr["bc_lo"] = ("noflux", "periodic")
    pr["bc_hi"] = ("dirichlet", "periodic")
    a = oracle.State(pr, phi, cs, cl)
    a.step(25)
    prT = dict(pr, n=(28, 20), bc_lo=pr["bc_lo"][::-1], bc_hi=pr["bc_hi"][::-1])
    b = oracle.State(prT, phi.T, cs.T, cl.T)
    b.step(25)
    for u, v in ((a.phi, b.phi), (a.cs, b.cs), (a.cl, b.cl)):
        assert np.abs(u - v.T).max() <= 1e-12


def test_mirror_symmetry_is_preserved():
    pr, phi, cs, cl = wl.random_state(2, (24, 20), A=1.5, b=0.3, seed=2)
    sym = lambda a: np.concatenate([a, a[::-1]], axis=0)   # mirror in y
    pr = dict(pr, n=(24, 40))
    st = oracle.State(pr, sym(phi), sym(cs), sym(cl))
    st.step(40)
    for u in (st.phi, st.cs, st.cl):
        assert np.abs(u - u[::-1]).max() <= 1e-12


def test_literal_form_agrees_with_conservative_form():
    """The literal c_s, c_l updates (Eqs. cs_nonvar, cl_nonvar with the source
    terms) and the conservative (c, d) updates differ by the discretisation
    error of the Stefan identity (Eq. model14) only: O(dt dx^2) per step."""
    errs = []
    for dx in (0.5, 0.25):
        n = int(16 / dx)
        pr = wl.scaled_params(1, (n,), dx, 0.1, 2.0, 0.1, A=0.4, b=0.3, a=0.2, dt=1e-4)
        x = (np.arange(n) + 0.5) * dx
        phi = wl.tanh_profile(x, 8.0)
        cs = 0.12 * (1 + 0.3 * np.sin(2 * np.pi * x / 16))
        cl = 1.1 + 0.25 * np.cos(2 * np.pi * x / 16)
        a = oracle.State(pr, phi, cs, cl)
        b = oracle.State(dict(pr, form="literal"), phi, cs, cl)
        a.step(10)
        b.step(10)
        errs.append(max(np.abs(a.cs - b.cs).max(), np.abs(a.cl - b.cl).max()))
    assert errs[1] < errs[0] / 2.5, errs


# --------------------------------------------------- brute force on tiny grids

BRUTE_CASES = [
    (1, (7,), dict(A=0.4, b=0.3, a=-0.3), 0),
    (1, (6,), dict(A=2.0, b=1.0, a=0.0, bc_lo=("noflux",), bc_hi=("dirichlet",), G_theta=0.05, x0=1.0,
                   v_pull=0.1), 40),
    (2, (6, 5), dict(A=0.4, b=0.3, a=0.2, lap=9), 0),
    (2, (5, 4), dict(A=1.5, b=0.3, a=0.0, lap=5, bc_lo=("noflux", "periodic"),
                     bc_hi=("dirichlet", "periodic")), 0),
    (3, (5, 4, 3), dict(A=0.4, b=0.3, a=-0.3, lap=19), 0),
    (3, (4, 4, 4), dict(A=0.0, b=0.5, a=0.0, lap=7, bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3,
                        interp="cubic", mobility="const"), 0),
    (3, (4, 3, 5), dict(A=2.0, b=1.0, a=0.0, lap=19, bc_lo=("noflux", "periodic", "dirichlet"),
                        bc_hi=("dirichlet", "periodic", "noflux"), G_theta=0.02), 0),
]


@pytest.mark.parametrize("dim,n,kw,step", BRUTE_CASES)
def test_rates_match_brute_force_evaluator(dim, n, kw, step):
    """The oracle's per-step rates (phidot, dc/dt, dd/dt) equal those of an
    independent literal evaluator (tests/bruteforce.py: the equations of the
    phase-field and concentration fluxes written out with Python loops over
    cells and faces) to rounding, on 3-7 cells per axis, for every stencil,
    boundary type, interpolation and mobility choice and a moving temperature.
    The convergence pin above fixes the continuum limit; this one fixes the
    discretisation itself (face means, one-sided normal and averaged transverse
    face gradients, the stencils, ghost rules)."""
    pr, phi, cs, cl = wl.random_state(dim, n, dx=0.5, seed=3 + step, **kw)
    st = oracle.State(pr, phi, cs, cl, step=step)
    got = st.rates()
    want = bruteforce.rates(pr, phi, cs, cl, t=step * pr["dt"])
    for name, a, b in zip(("phidot", "dc/dt", "dd/dt"), got, want):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (name, np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("plant", sorted(oracle.PLANT))
def test_planted_mistakes_break_the_brute_force_pin(plant):
    """Each planted mistake in the oracle moves its rates far from the literal
    evaluator's, so the agreement above is not a coincidence of the state."""
    pr, phi, cs, cl = wl.random_state(2, (6, 5), dx=0.5, seed=3, A=0.4, b=0.3, a=0.2, lap=9)
    want = bruteforce.rates(pr, phi, cs, cl)
    got = oracle.State(dict(pr, plant=plant), phi, cs, cl).rates()
    err = max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(got, want))
    assert err > 1e-6, (plant, err)


def test_thread_count_does_not_change_the_oracle():
    """oracle.set_threads (used for the one-thread CPU baseline) changes only
    how the sweeps are spread: every sweep writes each cell independently and
    the reductions sum in a fixed order, so one thread and all threads give
    the same bits."""
    pr, phi, cs, cl = wl.random_state(3, (20, 11, 9), A=1.5, b=0.3, seed=21)
    everyone = oracle.num_threads()
    out = []
    try:
        for n in (1, everyone):
            assert oracle.set_threads(n) == n
            st = oracle.State(pr, phi, cs, cl)
            st.step(5)
            out.append((st.phi.copy(), st.cs.copy(), st.cl.copy(), st.solute(), st.energy()))
    finally:
        oracle.set_threads(everyone)
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3] and out[0][4] == out[1][4]
