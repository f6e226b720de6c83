"""Thin-interface integrals and the partition law (asymptotics.py) against what
the mathematics fixes: the profile equation, exact symmetries, a closed-form
integral, an identity between G and F, linearity in A, and the limits of the
partition law."""
import math

import numpy as np
import pytest

from paper_2303_09671_gb300 import asymptotics as asy


def test_profile_solves_the_leading_order_equation():
    """phi_0' = -sqrt(2 f_dw(phi_0)) with f_dw = phi^2 (1-phi)^2 (Eq. sl5; the
    solid phi = 1 is at eta -> -inf, so the profile decreases)."""
    eta = np.linspace(-6, 6, 25)
    h = 1e-5
    d = (asy.phi0(eta + h) - asy.phi0(eta - h)) / (2 * h)
    f = asy.phi0(eta)
    np.testing.assert_allclose(d, -np.sqrt(2.0) * f * (1 - f), rtol=1e-8, atol=1e-12)
    assert asy.phi0(0.0) == 0.5


@pytest.mark.parametrize("a", [-1.0, 0.0, 0.7])
@pytest.mark.parametrize("r", [1e-4, 0.03])
def test_G_equal_for_b_one(a, r):
    """b = 1 gives h_n = p, antisymmetric about phi = 1/2 for any a, so the two
    half-line integrals of Eq. integral3 coincide."""
    gm, gp = asy.G_pm(r, 1.0, a)
    assert gm == pytest.approx(gp, rel=1e-10)
    assert asy.root_a(r, 1.0) == 0.0


def test_G_closed_form_quintic():
    """G^+ at b = 1, a = 0 is (1/r - 1) int_0^inf h(phi_0) d eta; with
    s = tanh(eta / sqrt 2) the integral is sqrt 2 int_0^1 h((1-s)/2)/(1-s^2) ds,
    done exactly."""
    sp = pytest.importorskip("sympy")
    s = sp.symbols("s")
    ph = (1 - s) / 2
    hq = ph ** 3 * (6 * ph ** 2 - 15 * ph + 10)
    exact = sp.sqrt(2) * sp.integrate(sp.cancel(hq / (1 - s ** 2)), (s, 0, 1))
    val = float(sp.N(exact, 30))
    r = 0.02
    gm, gp = asy.G_pm(r, 1.0, 0.0)
    assert gp == pytest.approx((1 / r - 1) * val, rel=1e-11)


def test_G_ratio_and_root_independent_of_mobility_ratio():
    """G^-/G^+ factor as (1/r - 1) times integrals of h_n alone, so the root
    a of G^- = G^+ does not depend on r = M_s/M_l."""
    b = 1e-3
    g1 = np.array(asy.G_pm(1e-4, b, 0.5))
    g2 = np.array(asy.G_pm(3e-4, b, 0.5))
    np.testing.assert_allclose(g1 / (1 / 1e-4 - 1), g2 / (1 / 3e-4 - 1), rtol=1e-10)
    a1, a2 = asy.root_a(1e-4, b), asy.root_a(3e-4, b)
    assert a1 is not None and a1 == pytest.approx(a2, abs=1e-9)
    gm, gp = asy.G_pm(1e-4, b, a1)
    assert gm == pytest.approx(gp, rel=1e-8)
    assert asy.qn_positive(1e-4, b, a1)


@pytest.mark.parametrize("r,b,a", [(1e-4, 1e-3, 0.0), (1e-4, 1e-3, 1.2), (3e-4, 0.3, -0.5), (0.01, 0.1, 0.4)])
@pytest.mark.parametrize("A", [0.0, 1.0, 2.0])
def test_delta_F_equals_G_identity(r, b, a, A):
    """Algebra of Eqs. integral1-3, normal2, interpolation1, shape_function
    (g = p): p~ = -(1 - h_n) + A (r - b) p (1 - h_n) / r and
    p - h_n = (1 - b) p (1 - h_n), so with antisymmetric p
        Delta F = D [1 - A (r - b) / (r (1 - b))],  D = (G^- - G^+) / (1/r - 1)
    for every a, b != 1.  In particular the a of G^- = G^+ makes Delta F = 0
    for every A."""
    gm, gp = asy.G_pm(r, b, a)
    D = (gm - gp) / (1.0 / r - 1.0)
    want = D * (1.0 - A * (r - b) / (r * (1.0 - b)))
    fm, fp = asy.F_pm(r, b, A, a)
    assert fm - fp == pytest.approx(want, rel=1e-8, abs=1e-10 * (abs(fm) + abs(fp) + 1e-3))


def test_delta_F_closed_form_b_one():
    """b = 1, a = 0 (quintic): Delta F = A (1/r - 1) int p (1 - p) d eta, the
    integral done exactly with s = tanh(eta / sqrt 2)."""
    sp = pytest.importorskip("sympy")
    s = sp.symbols("s")
    ph = (1 - s) / 2
    hq = ph ** 3 * (6 * ph ** 2 - 15 * ph + 10)
    exact = sp.sqrt(2) * sp.integrate(sp.cancel(hq * (1 - hq) / (1 - s ** 2)), (s, -1, 1))
    val = float(sp.N(exact, 30))
    r = 0.01
    for A in (0.5, 1.0, 2.0):
        assert asy.delta_F(r, 1.0, A) == pytest.approx(A * (1 / r - 1) * val, rel=1e-10)


def test_delta_F_linear_in_A():
    """Eq. integral2 is affine in A through (1 - A) a(phi)."""
    r, b = 0.01, 1.0
    d = [asy.delta_F(r, b, A) for A in (0.0, 0.5, 1.0, 2.0)]
    slope = d[2] - d[0]
    for A, v in zip((0.0, 0.5, 1.0, 2.0), d):
        assert v == pytest.approx(d[0] + A * slope, rel=1e-10, abs=1e-10)
    assert slope > 0   # more trapping with larger A


def test_partition_law_limits_and_slope():
    """Eq. partition1: k = k_e at V = 0, k -> 1 as V -> inf, increasing in V,
    and d ln k / dV = (1 - k_e) Delta F at V = 0 (W = D_l = 1)."""
    k_e, dF = 0.1, asy.delta_F(0.01, 1.0, 1.0)
    assert asy.k_of_V(0.0, k_e, dF) == k_e
    ks = asy.k_of_V(np.array([1e-3, 1e-2, 0.1, 1.0, 10.0, 100.0]), k_e, dF)
    assert np.all(np.diff(ks) > 0) and 1 - ks[-1] < 1e-3
    v = 1e-7
    slope = (math.log(asy.k_of_V(v, k_e, dF)) - math.log(k_e)) / v
    assert slope == pytest.approx((1 - k_e) * dF, rel=1e-5)
    with pytest.raises(ValueError):
        asy.k_of_V(0.1, k_e, -1.0)
