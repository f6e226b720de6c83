"""Thin-interface quantities of the model and the k(V) law they give (host).

These are the one-dimensional integrals of the paper's asymptotic analysis,
evaluated by quadrature over the leading-order phase-field profile, and the
partition law built from them:

* phi_0(eta) = [1 - tanh(eta / sqrt 2)] / 2, eta = x / W (supplement, Eq. sl6);
  solid (phi = 1) on the minus side, liquid on the plus side;
* 1/q_n = h_n/M_s + (1 - h_n)/M_l with h_n = b p / (b p + 1 - p)
  (Eqs. normal2, interpolation1), p = h + a (phi - 1/2) phi^2 (1 - phi)^2
  (Eq. interpolation2), g = p;
* a(phi) = (M_s - b M_l) p (1 - p) / (M_s (1 - p) + b M_l p) (Eq. shape_function);
* G^+- = M_l int_0^{+-inf} [1/q_n(phi_0) - 1/q_n^+-] d eta (Eq. integral3); the
  constant a of p is a root of G^- = G^+;
* F^+- = int_0^{+-inf} [p~(phi_0) - p~^+-] d eta, p~ = [g - 1 - (1-A) a(phi)] /
  (q_n / M_l) (Eqs. integral1, integral2), Delta F = F^- - F^+;
* ln(k_v / k_e) = (V W / D_l)(1 - k_v) Delta F (Eq. partition1), solved for k_v.

Algebra of these definitions (g = p, p antisymmetric about phi = 1/2):
p~ = -(1 - h_n) + A (r - b) p (1 - h_n) / r and p - h_n = (1 - b) p (1 - h_n),
whence Delta F = D [1 - A (r - b) / (r (1 - b))] with
D = (G^- - G^+) / (1/r - 1) = int (p - h_n) d eta for b != 1, and
Delta F = A (1/r - 1) int p (1 - p) d eta for b = 1.  So the a that makes
G^- = G^+ at b != 1 also makes Delta F vanish for every A: with that a the
partition law gives k = k_e at every V, and the law is informative only at
b = 1 (where G^- = G^+ for any a) or with a G^- != G^+.

Mobilities enter only through r = M_s / M_l.  For the dilute alloy at the
lowest order M_i = D_i c_i with c_s = k_e c_l, so r = k_e D_s / D_l.  In the
library's scaled units W = D_l = 1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

ETA_MAX = 40.0   # the integrands decay like exp(-sqrt(2) |eta|): negligible beyond


def phi0(eta):
    """Leading-order phase-field profile (Eq. sl6)."""
    return 0.5 * (1.0 - np.tanh(np.asarray(eta, dtype=float) / math.sqrt(2.0)))


def h_of(phi, interp="quintic"):
    phi = np.asarray(phi, dtype=float)
    if interp == "cubic":
        return phi * phi * (3.0 - 2.0 * phi)
    return phi ** 3 * (6.0 * phi * phi - 15.0 * phi + 10.0)


def p_of(phi, a=0.0, interp="quintic"):
    """p(phi) = h + a (phi - 1/2) phi^2 (1-phi)^2 (Eq. interpolation2)."""
    phi = np.asarray(phi, dtype=float)
    return h_of(phi, interp) + a * (phi - 0.5) * (phi * (1.0 - phi)) ** 2


def inv_qn(phi, r, b, a=0.0, interp="quintic"):
    """M_l / q_n(phi) with M_s / M_l = r (Eqs. normal2, interpolation1)."""
    p = p_of(phi, a, interp)
    hn = b * p / (b * p + 1.0 - p)
    return hn / r + (1.0 - hn)


def shape_a(phi, r, b, a=0.0, interp="quintic"):
    """a(phi) of Eq. shape_function with M_s / M_l = r."""
    p = p_of(phi, a, interp)
    return (r - b) * p * (1.0 - p) / (r * (1.0 - p) + b * p)


def _half_integral(g, side):
    """int_0^{+-inf} g(phi_0(eta)) d eta (side = +1 or -1; for -1 the integral
    runs from 0 down to -inf), taken over phi: d phi_0 / d eta =
    -sqrt(2) phi (1 - phi), so eta in (0, +inf) is phi in (0, 1/2) and eta in
    (-inf, 0) is phi in (1/2, 1), with the weight 1 / (sqrt 2 phi (1 - phi)).
    The integrands here vanish at the ends at least like phi^2 (1 - phi)^2, so
    the integral over phi is of a smooth function on a finite interval."""
    lo, hi = (0.0, 0.5) if side > 0 else (0.5, 1.0)
    val, _ = integrate.quad(lambda ph: g(ph) / (math.sqrt(2.0) * ph * (1.0 - ph)), lo, hi,
                            limit=400, epsabs=1e-14, epsrel=1e-12)
    return val if side > 0 else -val


def G_pm(r, b, a=0.0, interp="quintic"):
    """(G^-, G^+) of Eq. integral3, in units of W (M_l factored out)."""
    gp = _half_integral(lambda ph: inv_qn(ph, r, b, a, interp) - 1.0, +1)
    gm = _half_integral(lambda ph: inv_qn(ph, r, b, a, interp) - 1.0 / r, -1)
    return gm, gp


def qn_positive(r, b, a, interp="quintic"):
    """Whether q_n(phi) > 0 on [0, 1] (the paper's condition on b and a for the
    phase-concentration equations to be stable)."""
    ph = np.linspace(0.0, 1.0, 4001)
    with np.errstate(divide="ignore", invalid="ignore"):
        iq = inv_qn(ph, r, b, a, interp)
    return bool(np.all(np.isfinite(iq)) and iq.min() > 0.0)


def root_a(r, b, interp="quintic", step=0.05, a_max=20.0, rel_tol=1e-10):
    """The root of G^-(a) = G^+(a) closest to a = 0 (the paper picks among the
    smaller roots), searched outwards from 0 over the a for which q_n stays
    positive (|a| <= a_max); None if there is none.  For b = 1, h_n = p is antisymmetric about
    phi = 1/2 for every a, G^- = G^+ identically, and the answer is 0."""
    def D(a):
        gm, gp = G_pm(r, b, a, interp)
        return gm - gp, abs(gm) + abs(gp)

    d0, scale = D(0.0)
    if abs(d0) <= rel_tol * scale:
        return 0.0
    best = None
    for sgn in (+1.0, -1.0):
        a_prev, d_prev = 0.0, d0
        k = 1
        while True:
            a = sgn * k * step
            if abs(a) > a_max or not qn_positive(r, b, a, interp):
                break
            d, _ = D(a)
            if d_prev * d <= 0.0:
                lo, hi = sorted((a_prev, a))
                root = optimize.brentq(lambda x: D(x)[0], lo, hi, xtol=1e-13)
                if best is None or abs(root) < abs(best):
                    best = root
                break
            a_prev, d_prev = a, d
            k += 1
    return best


def p_tilde(phi, r, b, A, a=0.0, interp="quintic"):
    """p~(phi) of Eq. integral2 (g = p)."""
    g = p_of(phi, a, interp)
    return (g - 1.0 - (1.0 - A) * shape_a(phi, r, b, a, interp)) * inv_qn(phi, r, b, a, interp)


def F_pm(r, b, A, a=0.0, interp="quintic"):
    """(F^-, F^+) of Eq. integral1, in units of W."""
    lim_p = p_tilde(0.0, r, b, A, a, interp)   # liquid side, phi -> 0
    lim_m = p_tilde(1.0, r, b, A, a, interp)   # solid side, phi -> 1
    fp = _half_integral(lambda ph: p_tilde(ph, r, b, A, a, interp) - lim_p, +1)
    fm = _half_integral(lambda ph: p_tilde(ph, r, b, A, a, interp) - lim_m, -1)
    return fm, fp


def delta_F(r, b, A, a=0.0, interp="quintic"):
    fm, fp = F_pm(r, b, A, a, interp)
    return fm - fp


def k_of_V(V, k_e, dF, W=1.0, D_l=1.0):
    """k_v solving ln(k_v/k_e) = (V W / D_l)(1 - k_v) Delta F (Eq. partition1).

    For Delta F > 0 the root lies in (k_e, 1): the left side minus the right
    side is negative at k_e and positive at 1.  V = 0 gives k_e.
    """
    V = np.atleast_1d(np.asarray(V, dtype=float))
    out = np.empty_like(V)
    for i, v in enumerate(V):
        if v == 0.0:
            out[i] = k_e
            continue
        s = v * W / D_l * dF
        f = lambda k: math.log(k / k_e) - s * (1.0 - k)
        if s > 0:
            out[i] = optimize.brentq(f, k_e, 1.0, xtol=1e-15)
        else:
            raise ValueError("Delta F <= 0: no trapping root in (k_e, 1)")
    return out if out.size > 1 else float(out[0])
