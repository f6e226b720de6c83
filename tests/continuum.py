"""Continuum rates of the general model, derived symbolically from the free
energy functional, for pinning the oracle's discrete operators.

Independent of the specialised equations (Eqs. cs_nonvar, cl_nonvar,
phasefield_nonvar, drivingforce_nonvar) that the oracle implements: here the
rates are built from
  - the functional F = int H f_dw + sigma/2 |grad phi|^2 + f_s g + f_l (1-g)
    (Eq. model1.1) with the dilute free energies of Eq. dil_linear,
  - the flux laws of Eqs. model10-model11 (normal parts, with the Lagrange
    multiplier lambda) and the tangential laws J^t = -M^t grad_t(dF/dc),
  - the phase-field law of Eq. model12 with the sources S_s = S_l = -A(c_s - c_l),
  - the local solute balance of Eq. model14, which fixes lambda,
  - the interpolation choices of Sec. "Alternative choice of interpolation
    functions": M_s^n = M_s/h_n, M_l^n = M_l/(1-h_n) with h_n of Eq.
    interpolation1, M_s^t = M_s/p, M_l^t = M_l/(1-p), g = p (Eq. interpolation2),
  - the concentration laws of Eqs. model7-model8.
lambda and phi_t are solved pointwise from the 2x2 linear system of Eqs.
model12 and model14 (numerically, at each evaluation point).  Divergences are
taken with an 8th-order central difference of the numerically evaluated flux
(truncation ~1e-14 for the smooth manufactured fields used).
"""
from __future__ import annotations

import numpy as np
import sympy as sp

X, Y = sp.symbols("x y", real=True)
FD8 = np.array([1 / 280, -4 / 105, 1 / 5, -4 / 5, 0, 4 / 5, -1 / 5, 4 / 105, -1 / 280])


class ContinuumModel:
    def __init__(self, pr: dict, phi_e, cs_e, cl_e, t: float = 0.0, shifts: int = 0):
        """pr: the parameter dict; phi_e, cs_e, cl_e: sympy expressions in x, y."""
        self.pr = pr
        H, sig, Mphi = pr["H"], pr["sigma"], pr["M_phi"]
        Ds, Dl, ke, A, b, a = pr["D_s"], pr["D_l"], pr["k_e"], pr["A"], pr["b"], pr["a"]
        cubic = pr.get("interp", "quintic") == "cubic"
        const_mob = pr.get("mobility", "Dc") == "const"
        th = pr["theta_ref"] - pr["G_theta"] * ((X + shifts * pr["dx"] - pr["x0"]) - pr["v_pull"] * t)

        f = sp.Symbol("f")
        hf = f ** 2 * (3 - 2 * f) if cubic else f ** 3 * (6 * f ** 2 - 15 * f + 10)
        pf = hf + a * (f - sp.Rational(1, 2)) * f ** 2 * (1 - f) ** 2
        dpf = sp.diff(pf, f)
        csym, lsym = sp.symbols("cs cl", positive=True)
        # dilute ideal solution (scaled): f_i = f_i^A + eps_i c + c ln c - c,
        # eps_s - eps_l = -ln k_e (Eq. dil2), f_s^A - f_l^A = (k_e - 1) theta (Eq. dil5)
        fs_of = (ke - 1) * th + csym * sp.log(1 / sp.Float(ke)) + csym * sp.log(csym) - csym
        fl_of = lsym * sp.log(lsym) - lsym
        mus_of = sp.diff(fs_of, csym)
        mul_of = sp.diff(fl_of, lsym)

        ph, cs, cl = phi_e, cs_e, cl_e
        g = pf.subs(f, ph)
        dg = dpf.subs(f, ph)
        fs, fl = fs_of.subs(csym, cs), fl_of.subs(lsym, cl)
        mus, mul = mus_of.subs(csym, cs), mul_of.subs(lsym, cl)
        Ms = Ds if const_mob else Ds * cs
        Ml = Dl if const_mob else Dl * cl
        hn = b * g / (b * g + 1 - g)
        Msn, Mln = Ms / hn, Ml / (1 - hn)
        Mst, Mlt = Ms / g, Ml / (1 - g)
        S = -A * (cs - cl)
        ct = (cs - cl) + S * g + S * (1 - g)          # c~_s - c~_l
        gradphi = [sp.diff(ph, v) for v in (X, Y)]
        lapphi = sum(sp.diff(ph, v, 2) for v in (X, Y))
        dFdphi = H * sp.diff((f ** 2 * (1 - f) ** 2), f).subs(f, ph) - sig * lapphi + (fs - fl) * dg
        Es, El = mus * g, mul * (1 - g)               # dF/dc_s, dF/dc_l
        gEs = [sp.diff(Es, v) for v in (X, Y)]
        gEl = [sp.diff(El, v) for v in (X, Y)]
        args = (X, Y)
        L = lambda e: sp.lambdify(args, e, "numpy", cse=True)
        self._f = {k: L(v) for k, v in dict(
            phi=ph, cs=cs, cl=cl, g=g, dg=dg, dFdphi=dFdphi, Es=Es, El=El, Msn=Msn, Mln=Mln,
            Mst=Mst, Mlt=Mlt, S=S, ct=ct, gp0=gradphi[0], gp1=gradphi[1], gEs0=gEs[0],
            gEs1=gEs[1], gEl0=gEl[0], gEl1=gEl[1]).items()}
        self.Mphi = Mphi

    def _vals(self, x, y):
        return {k: np.broadcast_to(fn(x, y), np.broadcast(x, y).shape).astype(np.float64)
                for k, fn in self._f.items()}

    def _solve(self, x, y):
        """lambda and phi_t from Eqs. model12 and model14; fluxes J_s, J_l."""
        v = self._vals(x, y)
        gp = np.stack([v["gp0"], v["gp1"]])
        G2 = (gp ** 2).sum(0)
        Pe_s = gp * ((gp * np.stack([v["gEs0"], v["gEs1"]])).sum(0) / G2)   # P grad(dF/dc_s)
        Pe_l = gp * ((gp * np.stack([v["gEl0"], v["gEl1"]])).sum(0) / G2)
        ct, dg, Mphi = v["ct"], v["dg"], self.Mphi
        Msn, Mln = v["Msn"], v["Mln"]
        # J_s^n = -Msn [P grad Es - lam dg gp],  J_l^n = -Mln [P grad El + lam dg gp]
        # (i)  phit = -Mphi [dFdphi - lam ct dg + (S Es + S El) dg]
        # (ii) ct phit = -(J_s^n - J_l^n).gp
        #            = Msn (gp.PgEs) - Mln (gp.PgEl) - lam dg G2 (Msn + Mln)
        a_s = (gp * Pe_s).sum(0)
        a_l = (gp * Pe_l).sum(0)
        src = (v["S"] * v["Es"] + v["S"] * v["El"]) * dg
        # unknowns (lam, phit):
        #   Mphi(-ct dg) lam + phit = -Mphi (dFdphi + src)
        #   dg G2 (Msn+Mln) lam + ct phit = Msn a_s - Mln a_l
        a11, a12, r1 = -Mphi * ct * dg, np.ones_like(ct), -Mphi * (v["dFdphi"] + src)
        a21, a22, r2 = dg * G2 * (Msn + Mln), ct, Msn * a_s - Mln * a_l
        det = a11 * a22 - a12 * a21
        lam = (r1 * a22 - a12 * r2) / det
        phit = (a11 * r2 - a21 * r1) / det
        gEs = np.stack([v["gEs0"], v["gEs1"]])
        gEl = np.stack([v["gEl0"], v["gEl1"]])
        Jsn = -Msn * (Pe_s - lam * dg * gp)
        Jln = -Mln * (Pe_l + lam * dg * gp)
        Jst = -v["Mst"] * (gEs - Pe_s)
        Jlt = -v["Mlt"] * (gEl - Pe_l)
        return v, lam, phit, Jsn + Jst, Jln + Jlt

    def rates(self, x, y, h=1e-3):
        """(phi_t, c_t, d_t) at points (x, y) for c = g c_s + (1-g) c_l, d = c_s - c_l."""
        v, lam, phit, Js, Jl = self._solve(x, y)
        divs = np.zeros_like(phit)
        divl = np.zeros_like(phit)
        for ax in (0, 1):
            for w, k in zip(FD8, range(-4, 5)):
                if w == 0:
                    continue
                xx = x + (k * h if ax == 0 else 0.0)
                yy = y + (k * h if ax == 1 else 0.0)
                _, _, _, js, jl = self._solve(xx, yy)
                divs = divs + w * js[ax] / h
                divl = divl + w * jl[ax] / h
        cst = -divs + v["S"] * v["dg"] * phit                  # Eq. model7
        clt = -divl + v["S"] * v["dg"] * phit                  # Eq. model8
        ct = v["g"] * cst + (1 - v["g"]) * clt + (v["cs"] - v["cl"]) * v["dg"] * phit
        return phit, ct, cst - clt
