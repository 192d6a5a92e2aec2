"""Pins of the oracle's aligned-spin TaylorF2 coefficients at every PN order.

The stationary-phase phase of a quasi-circular inspiral follows from the binding energy
E(v) and the energy flux F(v) through d/dv[(1/(6 v^2)) dPsi/dv] = -E'(v)/F(v) (in units
of the total mass); the tests here derive the spin terms of the bracket that way, written
apart from the oracle, and compare them with the oracle's bracket:

  * spin-orbit (linear in the spins) at 1.5, 2.5, 3 and 3.5PN, for every mass ratio: the
    spin-orbit energy and flux of a circular orbit as collected by Blanchet (Living Rev.
    Relativ. 17 (2014) 2, Sec. 11.3): the 1.5/2.5PN terms (Blanchet, Buonanno & Faye
    2006), the 3PN tail term of the flux (Blanchet, Buonanno & Faye 2011), and the 3.5PN
    terms of the energy (Bohe, Marsat, Faye & Blanchet 2013) and flux (Bohe, Marsat &
    Blanchet 2013), with S_l = m1^2 chi1 + m2^2 chi2, Sigma_l = M (m2 chi2 - m1 chi1);
  * every spin term in the test-mass limit (eta -> 0), from physics that owes nothing to
    the PN two-body computation: the exact energy of a circular equatorial orbit of Kerr
    and the black-hole-perturbation flux of a particle on it (Tagoshi, Shibata, Tanaka &
    Sasaki 1996, to v^7);
  * the 3PN spin-spin terms for every mass ratio, against the per-body form of Bohe,
    Faye, Marsat & Porter (2015) with the black-hole quadrupole constant kappa = 1.

The oracle's model keeps spin-squared terms to 3PN and spin-linear terms to 3.5PN (the
3.5PN spin-squared tail and spin-cubed terms are left out on both sides), so the
comparisons stop there.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")
R = sp.Rational

V_TEST = [0.08, 0.15, 0.22, 0.3, 0.38]


def _bracket_from_energy_flux(e_norm, f_norm, v, Lv, order=8):
    """Solve d/dv[(1/(6 v^2)) dPsi/dv] = -E'/F for the TaylorF2 bracket, given the
    normalised energy e(v) (E = -(mu/2) v^2 e) and flux f(v) (F = (32/5) eta^2 v^10 f), both
    sympy series in v with ln v written as the symbol Lv.  Returns the bracket coefficients
    (p1 .. p4, c5 with phi5 = c5 (1 + 3 ln v), a6 + b6 ln v, p7) as a dict."""
    # -E'/F (32 eta / 5) v^9 = (v^2 e)' / (2 v f), independent of eta
    rhs = sp.expand(sp.series(sp.diff(v ** 2 * e_norm, v) / (2 * v * f_norm), v, 0, order).removeO())
    p1, p2, p3, p4, c5, a6, b6, p7 = syms = sp.symbols("p1 p2 p3 p4 c5 a6 b6 p7")
    lv = sp.log(v)
    bracket = 1 + p1 * v + p2 * v ** 2 + p3 * v ** 3 + p4 * v ** 4 + c5 * (1 + 3 * lv) * v ** 5 \
        + (a6 + b6 * lv) * v ** 6 + p7 * v ** 7
    # with Psi = (3 / (128 eta)) bracket / v^5 the factor (32 eta / 5) cancels eta
    psi = R(3, 128) * bracket / v ** 5
    lhs = sp.expand(sp.simplify(sp.diff(sp.diff(psi, v) / (6 * v ** 2), v) * R(32, 5) * v ** 9)).subs(lv, Lv)
    diff = sp.expand(lhs - rhs)
    eqs = []
    for n in range(order):
        cn = sp.expand(diff.coeff(v, n))
        eqs += [cn.coeff(Lv, 1), cn.coeff(Lv, 0)]
    sol = sp.solve([e for e in eqs if e != 0], list(syms), dict=True)
    assert len(sol) == 1
    return {str(k): sol[0][k] for k in syms}


def _oracle_spin_parts(v, m1, m2, c1, c2):
    """The oracle bracket's parts linear and quadratic in the spins at (c1, c2)."""
    b = oracle.pn_bracket(v, m1, m2, c1, c2)
    bm = oracle.pn_bracket(v, m1, m2, -c1, -c2)
    b0 = oracle.pn_bracket(v, m1, m2, 0.0, 0.0)
    return 0.5 * (b - bm), 0.5 * (b + bm) - b0


def _eval(expr, subs):
    return float(sp.N(expr.subs(subs), 30))


# ---------------------------------------------------------------------------------------
# spin-orbit terms from the PN energy and flux


def _spin_orbit_energy_flux(X1):
    """Normalised energy and flux of a circular orbit with aligned spins, terms linear in
    the spins to 3.5PN (plus the non-spinning terms that multiply them), at the exact
    mass fraction X1 = m1 / M.  The spins enter as eps * chi_i; eps tracks the order."""
    v, Lv, c1, c2, eps = sp.symbols("v Lv chi1 chi2 eps")
    pi, gE = sp.pi, sp.EulerGamma
    X1 = R(X1)
    X2 = 1 - X1
    eta, dl = X1 * X2, X1 - X2
    S = eps * (X1 ** 2 * c1 + X2 ** 2 * c2)       # S_l / M^2
    Sig = eps * (X2 * c2 - X1 * c1)               # Sigma_l / M^2
    x = v ** 2
    e = (1 + (-R(3, 4) - eta / 12) * x + (-R(27, 8) + R(19, 8) * eta - eta ** 2 / 24) * x ** 2
         + (-R(675, 64) + (R(34445, 576) - R(205, 96) * pi ** 2) * eta - R(155, 96) * eta ** 2
            - R(35, 5184) * eta ** 3) * x ** 3
         + v ** 3 * (R(14, 3) * S + 2 * dl * Sig)
         + v ** 5 * ((11 - R(61, 9) * eta) * S + dl * (3 - R(10, 3) * eta) * Sig)
         + v ** 7 * ((R(135, 4) - R(367, 4) * eta + R(29, 12) * eta ** 2) * S
                     + dl * (R(27, 4) - 39 * eta + R(5, 4) * eta ** 2) * Sig))
    f = (1 + (-R(1247, 336) - R(35, 12) * eta) * x + 4 * pi * v ** 3
         + (-R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2) * x ** 2
         + (-R(8191, 672) - R(583, 24) * eta) * pi * v ** 5
         + (R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE - R(856, 105) * (sp.log(16) + 2 * Lv)
            + (-R(134543, 7776) + R(41, 48) * pi ** 2) * eta - R(94403, 3024) * eta ** 2
            - R(775, 324) * eta ** 3) * v ** 6
         + (-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * pi * v ** 7
         + v ** 3 * (-4 * S - R(5, 4) * dl * Sig)
         + v ** 5 * ((-R(9, 2) + R(272, 9) * eta) * S + (-R(13, 16) + R(43, 4) * eta) * dl * Sig)
         + v ** 6 * (-16 * pi * S - R(31, 6) * pi * dl * Sig)
         + v ** 7 * ((R(476645, 6804) + R(6172, 189) * eta - R(2810, 27) * eta ** 2) * S
                     + (R(9535, 336) + R(1849, 126) * eta - R(1501, 36) * eta ** 2) * dl * Sig))
    return e, f, (v, Lv, c1, c2, eps)


@pytest.mark.parametrize("X1", [Fraction(1, 2), Fraction(3, 5), Fraction(7, 8), Fraction(19, 20)])
def test_spin_orbit_phase_follows_from_pn_energy_and_flux(X1):
    e, f, (v, Lv, c1, c2, eps) = _spin_orbit_energy_flux(X1)
    br = _bracket_from_energy_flux(e, f, v, Lv)
    # the part of each coefficient linear in the spins
    lin = {k: sp.expand(br[k]).coeff(eps, 1) for k in ("p3", "p4", "c5", "a6", "p7")}
    assert lin["p4"] == 0        # no spin-orbit term at 2PN
    m1, m2 = float(X1), 1.0 - float(X1)
    for ch1, ch2 in [(0.7, -0.4), (-0.3, 0.9), (0.05, 0.02)]:
        for vv in V_TEST:
            subs = {c1: ch1, c2: ch2}
            want = (_eval(lin["p3"], subs) * vv ** 3 + _eval(lin["c5"], subs) * (1 + 3 * math.log(vv)) * vv ** 5
                    + _eval(lin["a6"], subs) * vv ** 6 + _eval(lin["p7"], subs) * vv ** 7)
            got, _ = _oracle_spin_parts(vv, m1, m2, ch1, ch2)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (X1, ch1, ch2, vv, got, want)


def test_each_spin_orbit_order_is_checked_apart():
    """The comparison above sums the orders; recover each order's coefficient of the oracle
    from values at several v and compare it with the derivation, so that an error at one
    order cannot hide behind another at the same v."""
    X1 = Fraction(3, 4)
    e, f, (v, Lv, c1, c2, eps) = _spin_orbit_energy_flux(X1)
    br = _bracket_from_energy_flux(e, f, v, Lv)
    subs = {c1: 0.6, c2: -0.5}
    want = [_eval(sp.expand(br[k]).coeff(eps, 1), subs) for k in ("p3", "c5", "a6", "p7")]
    vs = np.array([0.05, 0.1, 0.15, 0.2, 0.25, 0.3])
    lin = np.array([_oracle_spin_parts(x, 0.75, 0.25, 0.6, -0.5)[0] for x in vs])
    A = np.column_stack([vs ** 3, vs ** 5 * (1 + 3 * np.log(vs)), vs ** 6, vs ** 7])
    got = np.linalg.lstsq(A, lin, rcond=None)[0]
    np.testing.assert_allclose(got, want, rtol=1e-6)


# ---------------------------------------------------------------------------------------
# test-mass limit: Kerr geodesic energy and the perturbative flux


@pytest.fixture(scope="module")
def kerr_bracket():
    v, u, qs, Lv = sp.symbols("v u q Lv")
    pi, gE = sp.pi, sp.EulerGamma
    # specific energy of a prograde circular equatorial orbit at u = sqrt(M / r)
    energy = (1 - 2 * u ** 2 + qs * u ** 3) / sp.sqrt(1 - 3 * u ** 2 + 2 * qs * u ** 3)
    # orbital frequency M Omega = u^3 / (1 + q u^3) = v^3: invert for u(v) order by order
    n = 10
    a = sp.symbols("a1:%d" % n)
    u_of_v = v + sum(a[i] * v ** (i + 2) for i in range(n - 2))
    rel = sp.series(u_of_v ** 3 / (1 + qs * u_of_v ** 3) - v ** 3, v, 0, n + 2).removeO()
    sol = {}
    for k in range(4, n + 2):
        ck = sp.expand(rel.coeff(v, k).subs(sol))
        free = [s for s in a if ck.has(s) and s not in sol]
        if free:
            sol[free[0]] = sp.solve(ck, free[0])[0]
    e_orb = sp.expand(sp.series(energy.subs(u, u_of_v.subs(sol)) - 1, v, 0, 12).removeO())
    e_norm = sp.expand(e_orb / (-v ** 2 / 2))
    # energy flux to infinity and into the horizon of a particle on that orbit, normalised
    # by the quadrupole flux (Tagoshi, Shibata, Tanaka & Sasaki 1996)
    f_norm = (1 - R(1247, 336) * v ** 2 + (4 * pi - R(11, 4) * qs) * v ** 3 + (-R(44711, 9072) + R(33, 16) * qs ** 2) * v ** 4
              + (-R(8191, 672) * pi - R(59, 16) * qs) * v ** 5
              + (R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE - R(856, 105) * (sp.log(16) + 2 * Lv)
                 - R(65, 6) * pi * qs + R(611, 504) * qs ** 2) * v ** 6
              + (-R(16285, 504) * pi + R(162035, 3888) * qs + R(65, 8) * pi * qs ** 2 - R(71, 24) * qs ** 3) * v ** 7)
    br = _bracket_from_energy_flux(e_norm, f_norm, v, Lv)
    return br, qs


def test_kerr_energy_reproduces_the_newtonian_and_1pn_binding_energy(kerr_bracket):
    br, qs = kerr_bracket
    # the non-spinning test-mass bracket is the eta -> 0 limit of the two-body one
    assert br["p2"] == R(3715, 756)
    assert sp.simplify(br["p3"].subs(qs, 0) + 16 * sp.pi) == 0


@pytest.mark.parametrize("chi", [0.9, 0.35, -0.6])
def test_spin_terms_in_the_test_mass_limit_follow_from_kerr(kerr_bracket, chi):
    """With m2 -> 0 every spin term of the bracket is fixed by the Kerr orbit and its flux.
    Linear terms are compared to 3.5PN, quadratic ones to 3PN (the model's orders)."""
    br, qs = kerr_bracket
    lin = {k: sp.expand(br[k]).coeff(qs, 1) for k in ("p3", "p4", "c5", "a6", "p7")}
    quad = {k: sp.expand(br[k]).coeff(qs, 2) for k in ("p3", "p4", "c5", "a6")}
    assert lin["p4"] == 0 and quad["p3"] == 0 and quad["c5"] == 0
    assert sp.expand(br["b6"]).coeff(qs, 1) == 0 and sp.expand(br["b6"]).coeff(qs, 2) == 0
    for vv in V_TEST:
        want_lin = chi * (float(lin["p3"]) * vv ** 3 + float(lin["c5"]) * (1 + 3 * math.log(vv)) * vv ** 5
                          + float(sp.N(lin["a6"])) * vv ** 6 + float(lin["p7"]) * vv ** 7)
        want_quad = chi * chi * (float(quad["p4"]) * vv ** 4 + float(quad["a6"]) * vv ** 6)
        # the secondary's spin must not matter: give it an arbitrary value
        got_lin, got_quad = _oracle_spin_parts(vv, 1.0, 0.0, chi, 0.0)
        assert abs(got_lin - want_lin) <= 1e-12 * max(1.0, abs(want_lin)), (vv, got_lin, want_lin)
        assert abs(got_quad - want_quad) <= 1e-12 * max(1.0, abs(want_quad)), (vv, got_quad, want_quad)
        b1 = oracle.pn_bracket(vv, 1.0, 0.0, chi, 0.8)
        b2 = oracle.pn_bracket(vv, 1.0, 0.0, chi, -0.3)
        assert abs(b1 - b2) <= 1e-13 * abs(b1)


# ---------------------------------------------------------------------------------------
# 3PN spin-spin terms: per-body form


def _per_body_3pn_spin_spin(X1, c1, c2):
    """3PN spin-spin phase coefficient of Bohe, Faye, Marsat & Porter (2015), written per
    body with the quadrupole constant kappa_i = 1 (black holes), plus the chi1 chi2 term."""
    X2 = 1 - X1
    eta = X1 * X2

    def self_term(X, c):
        qm = -R(410825, 672) - R(1085, 12) * X + R(1255, 36) * X ** 2      # kappa_i part
        ss = R(47035, 84) + R(2935, 6) * X - 120 * X ** 2                  # spin-squared part
        return X ** 2 * c ** 2 * (qm + ss)

    return self_term(X1, c1) + self_term(X2, c2) + eta * c1 * c2 * (R(32675, 112) + R(5575, 18) * eta)


def _spin_spin_2pn_khan(X1, c1, c2):
    """2PN spin-spin coefficient in the chi_s / chi_a form (Khan et al. 2016, App. B)."""
    X2 = 1 - X1
    eta, dl = X1 * X2, X1 - X2
    xs, xa = (c1 + c2) / 2, (c1 - c2) / 2
    return (-R(405, 8) + 200 * eta) * xa ** 2 - R(405, 4) * dl * xa * xs + (-R(405, 8) + R(5, 2) * eta) * xs ** 2


@pytest.mark.parametrize("X1", [Fraction(1, 2), Fraction(4, 7), Fraction(5, 6), Fraction(40, 41)])
def test_3pn_spin_spin_terms_equal_the_per_body_form(X1):
    X1 = R(X1)
    m1, m2 = float(X1), float(1 - X1)
    for ch1, ch2 in [(0.8, -0.7), (-0.2, -0.9), (0.5, 0.5)]:
        c1, c2 = R(ch1).limit_denominator(100), R(ch2).limit_denominator(100)
        s4 = float(_spin_spin_2pn_khan(X1, c1, c2))
        s6 = float(_per_body_3pn_spin_spin(X1, c1, c2))
        for vv in V_TEST:
            _, got = _oracle_spin_parts(vv, m1, m2, float(c1), float(c2))
            want = s4 * vv ** 4 + s6 * vv ** 6
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (X1, ch1, ch2, vv, got, want)
