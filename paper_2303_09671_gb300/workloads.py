"""Seeded synthetic inputs and scaled parameter sets.

This module holds the input recipe only: the scaled units, the parameter
values of the workloads and their seeded initial conditions.  It contains none
of the time-step arithmetic and is the one module shared by the CUDA path's
callers and the CPU oracle's callers.

Scaled units (supplement, non-dimensionalisation): length W, time W^2/D_l,
concentration c0 = c_inf, energy density R T_m c0 / V_m.  With W = sqrt(sigma/H)
(Eq. width) sigma = H; with gamma = I W H (Eq. energy, I = 1/(3 sqrt 2)) and the
capillary length d0 = gamma / [(R T_m / V_m) c_l^eq (1-k_e)^2] the well height is
H = theta (1-k_e)^2 / (I eps), eps = W/d0, theta = c_l^eq / c0 (liquidus slope
normalised to -1, Eq. dil7).  The phase-field mobility is M_phi = 1/(alpha H)
with alpha = tau D_l / W^2 and tau = 1/(M_phi H).

Fields are float64 numpy arrays shaped n[::-1] (x fastest).
"""
from __future__ import annotations

import math

import numpy as np

I_DW = 1.0 / (3.0 * math.sqrt(2.0))   # gamma = I W H for f_dw = phi^2 (1-phi)^2

DEFAULT_LAP = {1: 3, 2: 9, 3: 19}


def theta_from_undercooling(k_e: float, u: float) -> float:
    """c_l^eq / c0 at an undercooling u of the freezing range below the liquidus.

    Freezing range dT0 = |m| c0 (1-k_e)/k_e; T = T_L - u dT0 gives
    c_l^eq = c0 + u c0 (1-k_e)/k_e.
    """
    return 1.0 + u * (1.0 - k_e) / k_e


def effective_dmax(pr: dict, c_ref: float = 1.0, samples: int = 2001) -> float:
    """Largest diffusivity seen by the concentration equations (for the dt rule).

    Normal block: q_n (p/c_s + (1-p)/c_l); tangential: M_i/c_i; evaluated at the
    equilibrium pair c_s = k_e c_ref, c_l = c_ref over p in [0, 1].
    """
    cs, cl = pr["k_e"] * c_ref, c_ref
    if pr.get("mobility", "Dc") == "const":
        Ms, Ml = pr["D_s"], pr["D_l"]
    else:
        Ms, Ml = pr["D_s"] * cs, pr["D_l"] * cl
    p = np.linspace(0.0, 1.0, samples)
    b = pr["b"]
    Mbar = Ms * (1 - p) + b * Ml * p
    q = Ms * Ml * (b * p + 1 - p) / Mbar
    eig = q * (p / cs + (1 - p) / cl)
    return float(max(eig.max(), Ms / cs, Ml / cl))


def stable_dt(pr: dict) -> float:
    """Explicit-Euler step bound (the paper states none).

    dt_phi = 2 / (M_phi (lam sigma + 2 H)), dt_c = 2 / (lam D_max),
    lam = 4 dim / dx^2 (the nearest-neighbour bound, used for every stencil).
    """
    lam = 4.0 * pr["dim"] / pr["dx"] ** 2
    dt_phi = 2.0 / (pr["M_phi"] * (lam * pr["sigma"] + 2.0 * pr["H"]))
    dt_c = 2.0 / (lam * effective_dmax(pr))
    return min(dt_phi, dt_c)


def scaled_params(dim, n, dx, k_e, theta, D_s, *, A=0.4, b=None, a=0.0, eps=1.0,
                  alpha=1.0, lap=None, bc_lo=None, bc_hi=None, interp="quintic",
                  mobility="Dc", delta=1e-3, G_theta=0.0, v_pull=0.0, x0=0.0,
                  c_inf=1.0, shift=False, dt_factor=0.9, dt=None, form="cd"):
    """Parameter dict in scaled units (keys shared by the oracle and the library)."""
    H = theta * (1.0 - k_e) ** 2 / (I_DW * eps)
    n = tuple(int(v) for v in n)
    pr = dict(
        dim=dim, n=n, dx=float(dx),
        bc_lo=tuple(bc_lo or ("noflux",) * dim), bc_hi=tuple(bc_hi or ("noflux",) * dim),
        dirichlet=(0.0, k_e * c_inf, c_inf),
        interp=interp, lap=lap or DEFAULT_LAP[dim], mobility=mobility,
        H=H, sigma=H, M_phi=1.0 / (alpha * H), D_s=float(D_s), D_l=1.0, k_e=float(k_e),
        A=float(A), b=float(D_s if b is None else b), a=float(a), delta=float(delta),
        theta_ref=float(theta), G_theta=float(G_theta), v_pull=float(v_pull), x0=float(x0),
        c_inf=float(c_inf), shift=bool(shift), form=form, dt=0.0,
    )
    pr["dt"] = float(dt) if dt is not None else dt_factor * stable_dt(pr)
    return pr


def tanh_profile(x, x_front):
    """Equilibrium profile phi_0 = (1 - tanh((x - x_f)/(sqrt 2 W)))/2 (supplement Eq. eq18),
    evaluated as 1/(1 + exp(sqrt 2 (x - x_f))) so that the liquid-side tail keeps
    full relative precision."""
    u = np.sqrt(2.0) * (np.asarray(x, dtype=np.float64) - x_front)
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(u))


def cell_centres(n, dx):
    return (np.arange(n, dtype=np.float64) + 0.5) * dx


# ----------------------------------------------------------------- workloads

def planar_1d(N=1024, dx=0.25, k_e=0.1, u=0.3, D_s=1e-4, front_cell=256, **kw):
    """1D planar front: tanh profile centred at cell `front_cell`, solid at low x,
    c_s = k_e c0 and c_l = c0 everywhere, no-flux ends."""
    theta = theta_from_undercooling(k_e, u)
    pr = scaled_params(1, (N,), dx, k_e, theta, D_s, **kw)
    x = cell_centres(N, dx)
    phi = tanh_profile(x, front_cell * dx)
    cs = np.full(N, k_e * pr["c_inf"])
    cl = np.full(N, pr["c_inf"])
    return pr, phi, cs, cl


def perturbed_front_2d(nx=1024, ny=1024, dx=0.5, k_e=0.15, u=0.3, D_s=1e-3, front=128,
                       modes=8, amp_cells=2.0, seed=2, **kw):
    """2D planar front with a seeded sinusoidal perturbation.

    The growth axis is x (axis 0, no-flux); the front runs along y (periodic).
    Front position x_f(y) = front + sum_m a_m cos(2 pi k_m y / ny + psi_m) cells,
    k_m distinct integers in [1, min(64, ny/16)] (wavelengths of at least 16
    cells), amplitudes scaled so that max |x_f - front| = amp_cells.
    """
    rng = np.random.default_rng(seed)
    theta = theta_from_undercooling(k_e, u)
    kw.setdefault("bc_lo", ("noflux", "periodic"))
    kw.setdefault("bc_hi", ("noflux", "periodic"))
    pr = scaled_params(2, (nx, ny), dx, k_e, theta, D_s, **kw)
    kmax = max(1, min(64, ny // 16))
    ks = rng.choice(np.arange(1, kmax + 1), size=min(modes, kmax), replace=False)
    am = rng.uniform(0.5, 1.0, size=ks.size)
    ps = rng.uniform(0, 2 * math.pi, size=ks.size)
    yc = np.arange(ny)
    pert = (am[:, None] * np.cos(2 * math.pi * ks[:, None] * yc[None, :] / ny + ps[:, None])).sum(0)
    pert *= amp_cells / np.abs(pert).max()
    xf = (front + pert) * dx                          # per row y
    x = cell_centres(nx, dx)
    phi = tanh_profile(x[None, :], xf[:, None])       # shape (ny, nx)
    cs = np.full((ny, nx), k_e * pr["c_inf"])
    cl = np.full((ny, nx), pr["c_inf"])
    return pr, phi, cs, cl


def perturbed_front_3d(nx=64, ny=48, nz=40, dx=0.5, k_e=0.15, u=0.3, D_s=1e-3, front=20, modes=6,
                       amp_cells=2.0, seed=21, **kw):
    """3D planar front with a seeded perturbation: the 2D recipe above extruded
    to a second transverse axis.  Growth along x (no-flux); y and z periodic;
    x_f(y, z) = front + sum_m a_m cos(2 pi (k_m y / ny + l_m z / nz) + psi_m)
    cells with integer (k_m, l_m), wavelengths of at least 16 cells, scaled so
    that max |x_f - front| = amp_cells."""
    rng = np.random.default_rng(seed)
    theta = theta_from_undercooling(k_e, u)
    kw.setdefault("bc_lo", ("noflux", "periodic", "periodic"))
    kw.setdefault("bc_hi", ("noflux", "periodic", "periodic"))
    pr = scaled_params(3, (nx, ny, nz), dx, k_e, theta, D_s, **kw)
    ky = rng.integers(0, max(1, ny // 16) + 1, size=modes)
    kz = rng.integers(0, max(1, nz // 16) + 1, size=modes)
    kz[(ky == 0) & (kz == 0)] = 1
    am = rng.uniform(0.5, 1.0, size=modes)
    ps = rng.uniform(0, 2 * math.pi, size=modes)
    yy, zz = np.meshgrid(np.arange(ny), np.arange(nz), indexing="xy")      # shape (nz, ny)
    pert = sum(a * np.cos(2 * math.pi * (k * yy / ny + l * zz / nz) + q)
               for a, k, l, q in zip(am, ky, kz, ps))
    pert *= amp_cells / np.abs(pert).max()
    xf = (front + pert) * dx                                               # per (z, y)
    x = cell_centres(nx, dx)
    phi = tanh_profile(x[None, None, :], xf[:, :, None])                   # shape (nz, ny, nx)
    cs = np.full(phi.shape, k_e * pr["c_inf"])
    cl = np.full(phi.shape, pr["c_inf"])
    return pr, phi, cs, cl


def sphere_seed_3d(n=256, dx=0.5, k_e=0.1, u=0.5, D_s=1e-4, radius_cells=20.0, modes=8,
                   noise_cells=1.0, seed=3, **kw):
    """3D spherical solid seed with seeded surface noise at the box centre.

    R(nhat) = radius + sum_m b_m cos(k_m . nhat + psi_m) cells, k_m integer
    vectors with |k_m| <= 4, sum |b_m| = noise_cells; no-flux box.
    """
    rng = np.random.default_rng(seed)
    if np.isscalar(n):
        n = (n, n, n)
    theta = theta_from_undercooling(k_e, u)
    pr = scaled_params(3, n, dx, k_e, theta, D_s, **kw)
    ks = []
    while len(ks) < modes:
        k = rng.integers(-4, 5, size=3)
        if 0 < np.linalg.norm(k) <= 4:
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    bm = rng.uniform(0.2, 1.0, size=modes)
    bm *= noise_cells / bm.sum()
    ps = rng.uniform(0, 2 * math.pi, size=modes)
    nx_, ny_, nz_ = n
    phi = np.empty((nz_, ny_, nx_))
    xc = np.array([nx_, ny_, nz_], dtype=np.float64) * dx / 2
    x = cell_centres(nx_, dx) - xc[0]
    y = cell_centres(ny_, dx) - xc[1]
    for k in range(nz_):                      # plane by plane to bound memory
        z = (k + 0.5) * dx - xc[2]
        X, Y = np.meshgrid(x, y, indexing="xy")
        r = np.sqrt(X * X + Y * Y + z * z)
        rs = np.maximum(r, 1e-12)
        nh = np.stack([X / rs, Y / rs, np.full_like(X, z) / rs], -1)
        R = radius_cells + (bm * np.cos(nh @ ks.T + ps)).sum(-1)
        phi[k] = tanh_profile(r, R * dx)
    cs = np.full(phi.shape, k_e * pr["c_inf"])
    cl = np.full(phi.shape, pr["c_inf"])
    return pr, phi, cs, cl


def _smooth_field(rng, shape, dx, modes=4, kmax=3):
    """Sum of a few seeded low-wavenumber cosines over the grid, scaled to [-1, 1]."""
    dim = len(shape)
    axes = [np.arange(n, dtype=np.float64) / max(n, 1) for n in shape]   # (z,) y, x order
    out = np.zeros(shape)
    for _ in range(modes):
        ph = 0.0
        for a in range(dim):
            k = rng.integers(0, kmax + 1) if shape[a] > 1 else 0
            sh = [1] * dim
            sh[a] = shape[a]
            ph = ph + 2 * math.pi * k * axes[a].reshape(sh)
        out = out + rng.uniform(-1, 1) * np.cos(ph + rng.uniform(0, 2 * math.pi))
    m = np.abs(out).max()
    return out / m if m > 0 else out


def random_state(dim, n, dx=0.5, k_e=0.1, theta=2.0, D_s=0.1, seed=0, amp=0.3, wiggle=1.0, **kw):
    """Generic seeded non-equilibrium state on a small grid: a tanh front along x
    whose position is modulated (by `wiggle` cells) by the longest random modes
    across the front, in an undercooled melt (growth, no melt-back), and
    smooth positive random phase concentrations (mu_s != mu_l).  Used for parity
    and invariant tests."""
    rng = np.random.default_rng(seed)
    pr = scaled_params(dim, n, dx, k_e, theta, D_s, **kw)
    shape = tuple(int(v) for v in n[:dim][::-1])
    x = cell_centres(n[0], dx).reshape((1,) * (dim - 1) + (-1,))
    front = 0.5 * n[0] * dx
    if dim >= 2:
        mod = _smooth_field(rng, shape[:-1] + (1,), dx, kmax=1)
    else:
        mod = np.zeros((1,))
    phi = tanh_profile(x, front + wiggle * dx * mod)
    # c_l varies by k_e*amp only: the normal fluxes change c_s and c_l by the
    # same amount, so c_l variations must stay below c_s ~ k_e c_l
    cs = k_e * pr["c_inf"] * (1.0 + amp * _smooth_field(rng, shape, dx))
    cl = pr["c_inf"] * (1.0 + k_e * amp * _smooth_field(rng, shape, dx))
    return pr, phi, cs, cl


def pulled_front_1d(N=1024, dx=0.5, k_e=0.1, D_s=1e-4, V=0.1, G_theta=5.25e-3, front_cell=None,
                    **kw):
    """1D directional solidification in a frozen gradient with the moving window.

    theta(x,t) = theta_ref - G ((x - x0) - V t); the interface starts at x0 at the
    solidus of the alloy (theta_ref = 1/k_e, the reference of Sec. "Directional
    solidification"), solid at low x, no-flux cold end, Dirichlet hot end, and
    c_l = c_inf, c_s = k_e c_inf at every point (Sec. "Numerical technique").
    """
    front_cell = N // 4 if front_cell is None else front_cell
    x0 = front_cell * dx
    kw.setdefault("bc_lo", ("noflux",))
    kw.setdefault("bc_hi", ("dirichlet",))
    pr = scaled_params(1, (N,), dx, k_e, 1.0 / k_e, D_s, G_theta=G_theta, v_pull=V, x0=x0,
                       shift=True, **kw)
    x = cell_centres(N, dx)
    phi = tanh_profile(x, x0)
    cs = np.full(N, k_e * pr["c_inf"])
    cl = np.full(N, pr["c_inf"])
    return pr, phi, cs, cl


# ---------------------------------------------------------- physical units
# Table 1 of the paper (atomic per cent; SI otherwise): equilibrium partition
# coefficient, melting point [K], liquidus slope [K/%], alloy concentration
# [%], Gibbs-Thomson coefficient [K m], capillary length [m], liquid
# diffusivity [m^2/s], kinetic coefficient [s/m].
ALLOYS = {
    "Si-As": dict(k_e=0.3, T_m=1685.0, m=-4.0, c_inf=9.0, Gamma=3.4e-7, d0=13.5e-9, D_l=15e-9, beta=0.595),
    "Ni-Cu": dict(k_e=0.5, T_m=1728.0, m=-2.0, c_inf=5.0, Gamma=2.6e-7, d0=26e-9, D_l=3e-9, beta=0.2),
}


def physical_units(alloy, W=None):
    """Scales of the library's units for an alloy of Table 1: length W (default
    d_0, i.e. eps = W/d_0 = 1), time W^2/D_l, concentration c_inf, temperature
    |m| c_inf (theta = (T_m - T) / (|m| c_inf))."""
    a = ALLOYS[alloy]
    W = a["d0"] if W is None else float(W)
    return dict(length_m=W, time_s=W * W / a["D_l"], conc=a["c_inf"], temp_K=abs(a["m"]) * a["c_inf"],
                eps=W / a["d0"])


def physical_pulled_front(alloy, v_p, G, Ds_ratio, *, N=2048, dx=0.5, W=None, front_cell=None, **kw):
    """A pulled 1D front of a Table 1 alloy: pulling speed v_p [m/s], frozen
    gradient G [K/m], D_s/D_l, interface width W [m] (default d_0), converted to
    scaled units (V = v_p W / D_l, G_theta = G W / (|m| c_inf)); the start is that
    of pulled_front_1d (interface at the solidus of c_inf)."""
    a = ALLOYS[alloy]
    u = physical_units(alloy, W)
    V = v_p * u["length_m"] / a["D_l"]
    G_theta = G * u["length_m"] / u["temp_K"]
    pr, phi, cs, cl = pulled_front_1d(N=N, dx=dx, k_e=a["k_e"], D_s=Ds_ratio, V=V, G_theta=G_theta,
                                      front_cell=front_cell, eps=u["eps"], **kw)
    pr["units"] = u
    return pr, phi, cs, cl



def banding_front(v_p=0.3, *, A=1.0, b=1.0, N=8192, dx=0.5, front_cell=6000, theta_start=1.0, **kw):
    """A pulled Si-As front at the parameters of the paper's solute-band run
    (Sec. "Oscillations and solute bands": G = 1.4e6 K/m, D_s/D_l = 1e-3,
    v_p = 0.3 m/s; W = d_0), converted to scaled units by physical_pulled_front.
    The interface starts at theta = theta_start (the liquidus of c_inf at 1.0)
    instead of the solidus of c_inf, and far from the cold end of the window,
    so that the front reaches its steady position inside the window: the
    gradient of 5.25e-4 per W is too shallow for the solidus start."""
    pr, phi, cs, cl = physical_pulled_front("Si-As", v_p, 1.4e6, 1e-3, N=N, dx=dx, front_cell=front_cell,
                                            A=A, b=b, **kw)
    pr["theta_ref"] = float(theta_start)
    return pr, phi, cs, cl
