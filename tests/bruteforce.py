"""A literal evaluator of one explicit step's rates on tiny grids, written from
the equations with plain Python loops, for pinning the oracle's discretisation
(test infrastructure; it shares no code with the oracle or the CUDA path).

Discretisation (Sec. "Numerical technique": second-order finite differences on
a staggered grid, forward Euler), with the readings of the open points:
  * cell quantities: p = h + a (phi - 1/2) phi^2 (1-phi)^2 (Eq. interpolation2),
    mu_s = ln(c_s / k_e), mu_l = ln c_l (Eqs. dil5.1, dil5.2), Y = p mu_s +
    (1-p) mu_l, M_i = D_i c_i (or D_i for constant mobility);
  * gradients at cells: centred differences; Laplacian: 3-point (1D), 5- or
    9-point (2D), 7- or 19-point (3D);
  * phase-field rate (Eq. phasefield_nonvar with the driving force re-derived
    from the general model): phidot = R / K,
        K = 1/M_phi + (1-A)^2 d^2 b p (1-p) / (Mbar (b p + 1 - p)) r,
        R = sigma lap phi - H f_dw'(phi) - DeltaG p'
            + (1-A) d p (1-p) / Mbar (M_s grad mu_s - b M_l grad mu_l).grad phi r,
        DeltaG = f_s - f_l - mu_l d - D d (mu_s - mu_l),
        D = [M_s (1-p)(1 - A (1-p)) + A b M_l p^2] / Mbar,
        r = 1 / (|grad phi|^2 + delta^2), d = c_s - c_l;
  * faces: phi, c_s, c_l, d and phidot are the means of the two cells; p, M_s,
    M_l, Mbar, q = M_s M_l (b p + 1 - p) / Mbar, w_s = M_s (1-p) / Mbar,
    w_l = b M_l p / Mbar at those means; a gradient at a face has the one-sided
    difference as its normal component and the mean of the two cells' centred
    differences as its transverse components; with g = grad phi,
        F_s = q g (g.grad Y) r + M_s [grad mu_s - g (g.grad mu_s) r] + (1-A) d w_s phidot g r
        F_l = q g (g.grad Y) r + M_l [grad mu_l - g (g.grad mu_l) r] - (1-A) d w_l phidot g r
    (the brackets of Eqs. cs_nonvar, cl_nonvar, F = -J), F_c = p F_s + (1-p) F_l,
    F_d = F_s - F_l, and dc/dt, dd/dt = sum over axes of (F(+1/2) - F(-1/2)) / dx;
  * boundaries: a no-flux side mirrors the cells about the boundary face and
    has zero flux through it; a periodic axis wraps; a Dirichlet side holds
    fixed ghost cells with zero phase-field rate.
"""
import math

import numpy as np


def _h(pr, f):
    if pr.get("interp", "quintic") == "cubic":
        return f * f * (3 - 2 * f), 6 * f * (1 - f)
    return f ** 3 * (6 * f * f - 15 * f + 10), 30 * f * f * (1 - f) ** 2


def p_and_dp(pr, f):
    h, dh = _h(pr, f)
    a = pr["a"]
    g = f * (1 - f)
    # d/dphi [(phi - 1/2) g^2] = g^2 + 2 (phi - 1/2) g (1 - 2 phi)
    return h + a * (f - 0.5) * g * g, dh + a * (g * g + 2 * (f - 0.5) * g * (1 - 2 * f))


def mobilities(pr, cs, cl):
    if pr.get("mobility", "Dc") == "const":
        return pr["D_s"], pr["D_l"]
    return pr["D_s"] * cs, pr["D_l"] * cl


class Grid:
    """Index mapping of a tiny grid with its ghost cells."""

    def __init__(self, pr):
        self.pr = pr
        self.dim = pr["dim"]
        self.n = tuple(int(v) for v in pr["n"][: self.dim])

    def map(self, idx):
        """Interior index of a (possibly ghost) cell, or None for a Dirichlet ghost."""
        out = []
        for a, i in enumerate(idx):
            n = self.n[a]
            if 0 <= i < n:
                out.append(i)
                continue
            bc = self.pr["bc_lo"][a] if i < 0 else self.pr["bc_hi"][a]
            if bc == "dirichlet":
                return None
            if bc == "periodic":
                out.append(i % n)
            else:   # mirror about the boundary face
                out.append(-i - 1 if i < 0 else 2 * n - 1 - i)
        return tuple(out)

    def cells(self):
        return np.ndindex(*self.n)


def rates(pr, phi, cs, cl, t=0.0):
    """(phidot, dc/dt, dd/dt) at every cell; fields indexed [x, y, z] order
    reversed as in the library ([z][y][x]).  Loops over cells and faces."""
    G = Grid(pr)
    dim, dx = G.dim, pr["dx"]
    # fields indexed by (x, y, z) tuples
    F = {name: np.transpose(np.asarray(arr, dtype=np.float64)) for name, arr in
         (("phi", phi), ("cs", cs), ("cl", cl))}
    dphi, dcs, dcl = pr["dirichlet"]

    def val(name, idx):
        m = G.map(idx)
        if m is None:
            return {"phi": dphi, "cs": dcs, "cl": dcl}[name]
        return F[name][m]

    def cellq(idx):
        f, s, l = val("phi", idx), val("cs", idx), val("cl", idx)
        p, _ = p_and_dp(pr, f)
        mus, mul = math.log(s / pr["k_e"]), math.log(l)
        return {"phi": f, "cs": s, "cl": l, "mus": mus, "mul": mul, "Y": p * mus + (1 - p) * mul}

    def shift(idx, a, k):
        j = list(idx)
        j[a] += k
        return tuple(j)

    def cgrad(idx, key):
        return [(cellq(shift(idx, a, 1))[key] - cellq(shift(idx, a, -1))[key]) / (2 * dx) for a in range(dim)]

    def theta(idx):
        x = (idx[0] + 0.5) * dx
        return pr["theta_ref"] - pr["G_theta"] * ((x - pr["x0"]) - pr["v_pull"] * t)

    def laplacian(idx):
        f0 = cellq(idx)["phi"]
        lap = pr["lap"]

        def nb(*offs):
            j = list(idx)
            for a, k in offs:
                j[a] += k
            return cellq(tuple(j))["phi"] - f0

        faces = sum(nb((a, s)) for a in range(dim) for s in (-1, 1))
        if lap in (3, 5, 7):
            return faces / dx ** 2
        edges = sum(nb((a, s), (b, u)) for a in range(dim) for b in range(a + 1, dim)
                    for s in (-1, 1) for u in (-1, 1))
        if lap == 9:
            return (2.0 / 3.0 * faces + 1.0 / 6.0 * edges) / dx ** 2
        return (1.0 / 3.0 * faces + 1.0 / 6.0 * edges) / dx ** 2     # 19-point

    def phidot_interior(idx):
        q = cellq(idx)
        f, s, l = q["phi"], q["cs"], q["cl"]
        p, dp = p_and_dp(pr, f)
        Ms, Ml = mobilities(pr, s, l)
        b, A = pr["b"], pr["A"]
        Mbar = Ms * (1 - p) + b * Ml * p
        d = s - l
        gphi, gms, gml = cgrad(idx, "phi"), cgrad(idx, "mus"), cgrad(idx, "mul")
        r = 1.0 / (sum(g * g for g in gphi) + pr["delta"] ** 2)
        K = 1.0 / pr["M_phi"] + (1 - A) ** 2 * d * d * b * p * (1 - p) / (Mbar * (b * p + 1 - p)) * r
        th = theta(idx)
        f_s = -(1 - pr["k_e"]) * th + s * math.log(1 / pr["k_e"]) + s * math.log(s) - s
        f_l = l * math.log(l) - l
        D = (Ms * (1 - p) * (1 - A * (1 - p)) + A * b * Ml * p * p) / Mbar
        dG = f_s - f_l - q["mul"] * d - D * d * (q["mus"] - q["mul"])
        fdw1 = 2 * f * (1 - f) * (1 - 2 * f)
        cross = sum((Ms * gs - b * Ml * gl) * gp for gs, gl, gp in zip(gms, gml, gphi))
        R = (pr["sigma"] * laplacian(idx) - pr["H"] * fdw1 - dG * dp
             + (1 - A) * d * p * (1 - p) / Mbar * cross * r)
        return R / K

    pd_cache = {}

    def phidot(idx):
        m = G.map(idx)
        if m is None:
            return 0.0
        if m not in pd_cache:
            pd_cache[m] = phidot_interior(m)
        return pd_cache[m]

    def face_flux(L, a):
        """F_c, F_d through the face between cell L and its +a neighbour."""
        R_ = shift(L, a, 1)
        qL, qR = cellq(L), cellq(R_)
        f = 0.5 * (qL["phi"] + qR["phi"])
        s = 0.5 * (qL["cs"] + qR["cs"])
        l = 0.5 * (qL["cl"] + qR["cl"])
        d = s - l
        pdot = 0.5 * (phidot(L) + phidot(R_))
        p, _ = p_and_dp(pr, f)
        Ms, Ml = mobilities(pr, s, l)
        b, A = pr["b"], pr["A"]
        Mbar = Ms * (1 - p) + b * Ml * p
        qn = Ms * Ml * (b * p + 1 - p) / Mbar
        ws, wl = Ms * (1 - p) / Mbar, b * Ml * p / Mbar

        def fgrad(key):
            g = [0.0] * dim
            for c in range(dim):
                if c == a:
                    g[c] = (qR[key] - qL[key]) / dx
                else:
                    g[c] = 0.5 * (cgrad(L, key)[c] + cgrad(R_, key)[c])
            return g

        g, gY, gs, gl = fgrad("phi"), fgrad("Y"), fgrad("mus"), fgrad("mul")
        r = 1.0 / (sum(x * x for x in g) + pr["delta"] ** 2)
        dot = lambda u, v: sum(x * y for x, y in zip(u, v))
        Fs = qn * g[a] * dot(g, gY) * r + Ms * (gs[a] - g[a] * dot(g, gs) * r) + (1 - A) * d * ws * pdot * g[a] * r
        Fl = qn * g[a] * dot(g, gY) * r + Ml * (gl[a] - g[a] * dot(g, gl) * r) - (1 - A) * d * wl * pdot * g[a] * r
        return p * Fs + (1 - p) * Fl, Fs - Fl

    def flux(L, a):
        """Zero through a no-flux boundary face."""
        i = L[a]
        if (i == -1 and pr["bc_lo"][a] == "noflux") or (i == G.n[a] - 1 and pr["bc_hi"][a] == "noflux"):
            return 0.0, 0.0
        return face_flux(L, a)

    shape = G.n
    out = [np.zeros(shape) for _ in range(3)]
    for idx in G.cells():
        out[0][idx] = phidot(idx)
        dc = dd = 0.0
        for a in range(dim):
            cp, dp_ = flux(idx, a)
            cm, dm = flux(shift(idx, a, -1), a)
            dc += (cp - cm) / dx
            dd += (dp_ - dm) / dx
        out[1][idx] = dc
        out[2][idx] = dd
    return tuple(np.transpose(o) for o in out)
