"""Pins of the oracle's waveform, PSD, masses and detector response.

The paper prints no waveform formula (it uses IMRPhenom models, Sec. III); the TaylorF2
phase and f^(-7/6) amplitude are tied here to physics they must reproduce:
  * the non-spinning phase coefficients follow from the post-Newtonian binding energy and
    flux by the stationary-phase relation d/dv[(1/(6 v^2)) dPsi/dv] = -E'(v)/F(v);
  * the 1.5PN / 2PN spin terms, written in the oracle in (beta, sigma) form, equal the
    chi_s / chi_a form;
  * in the test-mass limit the secondary's spin drops out of every spin term;
  * relabelling the two bodies leaves the phase unchanged;
  * the amplitude equals the stationary-phase transform of the quadrupole chirp, which
    this test computes by an FFT of a numerically generated time-domain chirp.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC
import workloads

T_SUN = 4.925490947641267e-6
MPC_S = 3.0856775814913673e22 / 299792458.0


def par(mc=20.0, q=1.5, chi1=0.2, chi2=-0.3, ra=1.0, dec=0.3, psi=0.4, iota=0.7, dl=400.0, tc=0.0, phic=0.0):
    return np.array([mc, q, chi1, chi2, ra, dec, psi, iota, dl, tc, phic], dtype=np.float64)


def test_psd_knee_value_and_positivity():
    # at x = f/215 Hz = 1 the bracket is 1 - 5 + 111 * (1/2) / (3/2) = 33
    assert abs(oracle.psd_aligo(215.0)[0] / 3.3e-48 - 1) < 1e-13
    f = np.linspace(20, 1024, 5000)
    assert np.all(oracle.psd_aligo(f) > 0)


def test_component_masses_round_trip():
    for m1, m2 in [(30.0, 25.0), (1.9, 1.2), (80.0, 10.0)]:
        mc = (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2
        a, b = oracle.component_masses(mc, m1 / m2)
        assert abs(a - m1) < 1e-12 * m1 and abs(b - m2) < 1e-12 * m2


def test_mass_jacobian_against_finite_difference_determinant():
    mc, q, h = 12.0, 2.3, 1e-6
    def m(x, y):
        return np.array(oracle.component_masses(x, y))
    J = np.column_stack([(m(mc + h, q) - m(mc - h, q)) / (2 * h), (m(mc, q + h) - m(mc, q - h)) / (2 * h)])
    assert abs(abs(np.linalg.det(J)) / oracle.mass_jacobian(mc, q) - 1) < 1e-8


def test_isco_frequency_of_the_tiny_workload():
    mc = (30 * 25) ** 0.6 / 55 ** 0.2
    f = oracle.f_isco(mc, 1.2)
    assert abs(f - 79.9486) < 1e-3
    # 240 live bins on the 20 Hz + k * 0.25 Hz grid
    k = np.arange(1969)
    assert np.sum(20 + 0.25 * k < f) == 240


# ---------------------------------------------------------------------------------------
# TaylorF2 phase coefficients


def _energy_flux_coefficients():
    """Non-spinning TaylorF2 coefficients implied by the 3PN energy and 3.5PN flux of a
    circular orbit (Blanchet, Living Rev. Relativ. 17 (2014) 2, Eqs. 233 and 314), as
    sympy expressions in eta; the 2.5PN constant is the (1 + 3 ln v) convention."""
    sp = pytest.importorskip("sympy")
    v, eta, Lv = sp.symbols("v eta Lv", positive=True)
    pi, gE = sp.pi, sp.EulerGamma
    R = sp.Rational
    x = v ** 2
    E = -(eta * v ** 2 / 2) * (1 + (-R(3, 4) - eta / 12) * x + (-R(27, 8) + R(19, 8) * eta - eta ** 2 / 24) * x ** 2
                               + (-R(675, 64) + (R(34445, 576) - R(205, 96) * pi ** 2) * eta - R(155, 96) * eta ** 2
                                  - R(35, 5184) * eta ** 3) * x ** 3)
    F = R(32, 5) * eta ** 2 * v ** 10 * (
        1 + (-R(1247, 336) - R(35, 12) * eta) * x + 4 * pi * v ** 3
        + (-R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2) * x ** 2
        + (-R(8191, 672) - R(583, 24) * eta) * pi * v ** 5
        + (R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE - R(856, 105) * (sp.log(16) + 2 * Lv)
           + (-R(134543, 7776) + R(41, 48) * pi ** 2) * eta - R(94403, 3024) * eta ** 2 - R(775, 324) * eta ** 3) * v ** 6
        + (-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * pi * v ** 7)
    rhs = sp.series(sp.expand(-sp.diff(E, v) / F * (32 * eta / 5) * v ** 9), v, 0, 8).removeO()
    # unknown TaylorF2 coefficients; phi5 = c5 (1 + 3 ln v), phi6 = a6 + b6 ln v
    p2, p3, p4, c5, a6, b6, p7, p1 = sp.symbols("p2 p3 p4 c5 a6 b6 p7 p1")
    lv = sp.log(v)
    bracket = 1 + p1 * v + p2 * v ** 2 + p3 * v ** 3 + p4 * v ** 4 + c5 * (1 + 3 * lv) * v ** 5 + (a6 + b6 * lv) * v ** 6 \
        + p7 * v ** 7
    psi = R(3, 128) / eta * bracket / v ** 5
    lhs = sp.diff(sp.diff(psi, v) / (6 * v ** 2), v) * (32 * eta / 5) * v ** 9
    lhs = sp.expand(sp.simplify(lhs)).subs(sp.log(v), Lv)
    diff = sp.expand(lhs - rhs)
    eqs = []
    for n in range(0, 8):
        cn = diff.coeff(v, n)
        eqs += [sp.expand(cn).coeff(Lv, 1), sp.expand(cn).coeff(Lv, 0)]
    sol = sp.solve([e for e in eqs if e != 0], [p1, p2, p3, p4, c5, a6, b6, p7], dict=True)
    assert len(sol) == 1
    return sp, v, eta, sol[0], (p1, p2, p3, p4, c5, a6, b6, p7)


def test_nonspinning_phase_follows_from_pn_energy_and_flux():
    sp, v, eta, sol, syms = _energy_flux_coefficients()
    p1, p2, p3, p4, c5, a6, b6, p7 = syms
    for m1, m2 in [(1.4, 1.3), (30.0, 25.0), (40.0, 8.0)]:
        e = m1 * m2 / (m1 + m2) ** 2
        co = {s: float(sol[s].subs(eta, e)) for s in syms}
        for vv in [0.08, 0.2, 0.35]:
            ref = (1 + co[p1] * vv + co[p2] * vv ** 2 + co[p3] * vv ** 3 + co[p4] * vv ** 4
                   + co[c5] * (1 + 3 * math.log(vv)) * vv ** 5 + (co[a6] + co[b6] * math.log(vv)) * vv ** 6
                   + co[p7] * vv ** 7)
            got = oracle.pn_bracket(vv, m1, m2, 0.0, 0.0)
            assert abs(got / ref - 1) < 1e-12, (m1, m2, vv)


def _chis_chia_low_order_spin(eta, delta, chis, chia):
    """1.5PN and 2PN spin terms in the chi_s / chi_a form (Khan et al. 2016, App. B)."""
    s3 = 113.0 / 3 * delta * chia + (113.0 / 3 - 76.0 * eta / 3) * chis
    s4 = (-405.0 / 8 + 200 * eta) * chia ** 2 - 405.0 / 4 * delta * chia * chis + (-405.0 / 8 + 5 * eta / 2) * chis ** 2
    return s3, s4


def test_low_order_spin_terms_agree_with_chis_chia_form():
    for m1, m2, c1, c2 in [(1.5, 1.2, 0.04, -0.03), (30.0, 25.0, 0.3, -0.1), (60.0, 12.0, -0.7, 0.8)]:
        M = m1 + m2
        eta, delta = m1 * m2 / M ** 2, (m1 - m2) / M
        chis, chia = 0.5 * (c1 + c2), 0.5 * (c1 - c2)
        s3, s4 = _chis_chia_low_order_spin(eta, delta, chis, chia)
        # the spin part of the bracket is exactly s3 v^3 + s4 v^4 + s5 (1 + 3 ln v) v^5
        # + s6 v^6 + s7 v^7: recover the five coefficients from five values of v
        vs = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
        d = np.array([oracle.pn_bracket(v, m1, m2, c1, c2) - oracle.pn_bracket(v, m1, m2, 0.0, 0.0) for v in vs])
        A = np.column_stack([vs ** 3, vs ** 4, vs ** 5 * (1 + 3 * np.log(vs)), vs ** 6, vs ** 7])
        a, b = np.linalg.solve(A, d)[:2]
        assert abs(a - s3) < 1e-9 * max(1, abs(s3))
        assert abs(b - s4) < 1e-9 * max(1, abs(s4))


def test_spin_terms_lose_the_secondary_spin_in_the_test_mass_limit():
    m1, m2 = 1.0, 1e-9
    for v in [0.1, 0.3, 0.5]:
        a = oracle.pn_bracket(v, m1, m2, 0.6, -0.9)
        b = oracle.pn_bracket(v, m1, m2, 0.6, 0.4)
        assert abs(a - b) < 1e-6 * abs(a)
        c = oracle.pn_bracket(v, m1, m2, -0.6, 0.4)
        assert abs(a - c) > 1e-3 * abs(a)      # the primary's spin does matter


def test_phase_is_invariant_under_relabelling_the_bodies():
    f = np.array([20.0, 55.5, 130.0])
    a = par(mc=14.0, q=2.5, chi1=0.5, chi2=-0.2, tc=0.01, phic=1.0)
    b = a.copy()
    b[Q], b[CHI1], b[CHI2] = 1 / a[Q], a[CHI2], a[CHI1]
    np.testing.assert_allclose(oracle.taylorf2_phase(f, a), oracle.taylorf2_phase(f, b), rtol=1e-13, atol=1e-9)


def test_phase_derivative_is_two_pi_time_to_coalescence_at_leading_order():
    # dPsi/df = 2 pi (t_c - tau(f)) with tau the Newtonian time to coalescence; at very low
    # v the PN corrections vanish, so compare at a tiny frequency with high relative accuracy
    p = par(mc=1.2, q=1.0, chi1=0.0, chi2=0.0, tc=0.0)
    f, h = 0.5, 1e-6
    d = (oracle.taylorf2_phase([f + h], p)[0] - oracle.taylorf2_phase([f - h], p)[0]) / (2 * h)
    tau = 5.0 / 256 * (math.pi * f) ** (-8.0 / 3) * (p[MC] * T_SUN) ** (-5.0 / 3)
    assert abs(d / (-2 * math.pi * tau) - 1) < 2e-2


# ---------------------------------------------------------------------------------------
# amplitude


def test_amplitude_matches_fft_of_the_quadrupole_chirp():
    """|h+(f)| of a face-on source equals the transform of the time-domain Newtonian chirp
    h(t) = (4/d) Mc^(5/3) (pi f(t))^(2/3) cos Phi(t), generated numerically here.  A light
    chirp (Mc = 2 Msun) keeps fdot/f^2 below 0.004 in band, where the stationary-phase
    approximation itself is accurate to a fraction of a percent."""
    mc_s = 2.0 * T_SUN
    d_s = 1.0 * MPC_S
    fs, T = 4096.0, 32.0
    t = np.arange(int(fs * T)) / fs
    tc = 28.0
    tau = np.clip(tc - t, 1e-4, None)
    f_t = (1 / math.pi) * (5.0 / (256.0 * tau)) ** 0.375 * mc_s ** (-0.625)
    phi = -2.0 * (tau / (5 * mc_s)) ** 0.625
    h = 4.0 / d_s * mc_s ** (5.0 / 3) * (math.pi * f_t) ** (2.0 / 3) * np.cos(phi)
    w = ((f_t > 30) & (f_t < 400)).astype(float)
    on = (f_t >= 29) & (f_t <= 30)
    w[on] = 0.5 * (1 - np.cos(math.pi * (f_t[on] - 29)))
    off = (f_t >= 400) & (f_t < 600)
    w[off] = 0.5 * (1 + np.cos(math.pi * (f_t[off] - 400) / 200))
    w[t >= tc] = 0.0
    hf = np.fft.rfft(h * w) / fs
    freqs = np.fft.rfftfreq(len(t), 1 / fs)
    band = (freqs > 45) & (freqs < 150)
    p = par(mc=2.0, q=1.0, chi1=0.0, chi2=0.0, iota=0.0, dl=1.0)
    hp, _ = oracle.polarisations(freqs[band], p)
    ratio = np.abs(hf[band]) / np.abs(hp)
    # the SPA ripples average out over a few bins
    k = 64
    sm = np.convolve(ratio, np.ones(k) / k, mode="valid")
    assert np.all(np.abs(sm - 1) < 0.01), (sm.min(), sm.max())


def test_flat_psd_norm_has_the_closed_form():
    """4 df sum |h+|^2 / S0 over the grid = (3 A^2 / S0)(f_lo^(-4/3) - f_hi^(-4/3)) + Euler-
    Maclaurin end corrections, and is independent of every phase parameter."""
    f_lo, df, n = 20.0, 0.25, 1969
    f = f_lo + df * np.arange(n)
    f_hi = f[-1]
    S0 = 1e-46
    p = par(mc=1.2, q=1.2, chi1=0.03, chi2=0.01, iota=0.0, dl=100.0)
    hp, _ = oracle.polarisations(f, p)
    got = 4 * df * np.sum(np.abs(hp) ** 2) / S0
    A = oracle.amplitude(p[MC], p[DL])
    g = lambda x: x ** (-7.0 / 3)
    gp = lambda x: -7.0 / 3 * x ** (-10.0 / 3)
    g3 = lambda x: (-7.0 / 3) * (-10.0 / 3) * (-13.0 / 3) * x ** (-16.0 / 3)
    integral = 0.75 * (f_lo ** (-4.0 / 3) - f_hi ** (-4.0 / 3))
    em = integral + df / 2 * (g(f_lo) + g(f_hi)) + df ** 2 / 12 * (gp(f_hi) - gp(f_lo)) \
        - df ** 4 / 720 * (g3(f_hi) - g3(f_lo))
    ref = 4 * A * A / S0 * em
    assert abs(got / ref - 1) < 1e-10
    for tc, phic, chi1 in [(0.02, 1.0, -0.04), (-0.5, 4.0, 0.0)]:
        p2 = p.copy()
        p2[TC], p2[PHIC], p2[CHI1] = tc, phic, chi1
        hp2, _ = oracle.polarisations(f, p2)
        assert abs(4 * df * np.sum(np.abs(hp2) ** 2) / S0 / got - 1) < 1e-13


def test_cross_polarisation_is_a_quarter_cycle_behind():
    f = np.array([30.0, 60.0])
    p = par(iota=0.0)
    hp, hc = oracle.polarisations(f, p)
    np.testing.assert_allclose(hc, -1j * hp, rtol=1e-14)


def test_waveform_vanishes_at_and_above_isco():
    p = par(mc=40.0, q=1.0)
    fi = oracle.f_isco(p[MC], p[Q])
    hp, hc = oracle.polarisations(np.array([fi * 0.999, fi, fi * 1.5]), p)
    assert hp[0] != 0 and hp[1] == 0 and hp[2] == 0 and hc[1] == 0


# ---------------------------------------------------------------------------------------
# detector response


def test_detector_geometry_inputs_are_orthonormal():
    for name, d in workloads.DETECTORS.items():
        x, y = np.array(d["xarm"]), np.array(d["yarm"])
        assert abs(np.linalg.norm(x) - 1) < 1e-9 and abs(np.linalg.norm(y) - 1) < 1e-9
        # surveyed arms: orthogonal to the precision of the published geometry
        assert abs(x @ y) < 1e-6


def _orthonormal_arms(name):
    d = workloads.DETECTORS[name]
    x = np.array(d["xarm"]) / np.linalg.norm(d["xarm"])
    y = np.array(d["yarm"]) - (np.array(d["yarm"]) @ x) * x
    return x, y / np.linalg.norm(y)


def _radec_of(n):
    n = n / np.linalg.norm(n)
    return math.atan2(n[1], n[0]) % (2 * math.pi), math.asin(n[2])


@pytest.mark.parametrize("name", ["H1", "L1", "V1"])
def test_antenna_special_directions(name):
    x, y = _orthonormal_arms(name)
    # zenith of the detector plane: F+^2 + Fx^2 = 1 for every psi
    ra, dec = _radec_of(np.cross(x, y))
    for psi in [0.0, 0.3, 1.2, 2.9]:
        fp, fc = oracle.antenna(x, y, ra, dec, psi, 0.0)
        assert abs(fp * fp + fc * fc - 1) < 1e-12
    # along an arm: 1/4; along the in-plane bisector: 0
    ra, dec = _radec_of(x)
    fp, fc = oracle.antenna(x, y, ra, dec, 0.7, 0.0)
    assert abs(fp * fp + fc * fc - 0.25) < 1e-12
    ra, dec = _radec_of(x + y)
    fp, fc = oracle.antenna(x, y, ra, dec, 0.7, 0.0)
    assert abs(fp * fp + fc * fc) < 1e-12


def test_antenna_psi_invariance_bound_and_sidereal_shift():
    d = workloads.DETECTORS["L1"]
    x, y = np.array(d["xarm"]), np.array(d["yarm"])
    rng = np.random.default_rng(5)
    for _ in range(50):
        ra, dec = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        vals = []
        for psi in rng.uniform(0, math.pi, 4):
            fp, fc = oracle.antenna(x, y, ra, dec, psi, 0.4)
            assert abs(fp) <= 1 and abs(fc) <= 1
            vals.append(fp * fp + fc * fc)
        assert np.ptp(vals) < 1e-13
        g = rng.uniform(0, 6)
        a = oracle.antenna(x, y, ra, dec, 0.5, 0.4)
        b = oracle.antenna(x, y, ra + g, dec, 0.5, 0.4 + g)
        np.testing.assert_allclose(a, b, atol=1e-13)


def test_time_delays_and_light_travel_time():
    rh, rl = np.array(workloads.DETECTORS["H1"]["vertex"]), np.array(workloads.DETECTORS["L1"]["vertex"])
    light = np.linalg.norm(rh - rl) / 299792458.0
    assert abs(light - 10.01e-3) < 0.02e-3
    ra, dec = _radec_of(rl - rh)   # source along the baseline, beyond L1
    dt = oracle.time_delay(rh, ra, dec, 0.0) - oracle.time_delay(rl, ra, dec, 0.0)
    assert abs(dt - light) < 1e-12
    rng = np.random.default_rng(9)
    for _ in range(100):
        ra, dec = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        assert abs(oracle.time_delay(rh, ra, dec, 0.3) - oracle.time_delay(rl, ra, dec, 0.3)) <= light + 1e-15


def test_detector_strain_is_the_projected_waveform_delayed_in_time():
    """h_det(f; t_c) = F+ h+(f; t_c + dt) + Fx hx(f; t_c + dt): the detector delay acts as a
    later coalescence time, with the same sign convention as t_c inside Psi."""
    v, xa, ya = workloads.network(["H1", "V1"])
    n = 64
    ev = oracle.OracleEvent(20.0, 1.0, n, np.ones((2, n)), v, xa, ya, gmst=0.9)
    p = par()
    f = ev.freqs()
    for d in range(2):
        h = oracle.detector_strain(ev, d, f, p)
        fp, fc = oracle.antenna(xa[d], ya[d], p[RA], p[DEC], p[PSI], 0.9)
        dt = oracle.time_delay(v[d], p[RA], p[DEC], 0.9)
        q = p.copy()
        q[TC] += dt
        hp, hc = oracle.polarisations(f, q)
        np.testing.assert_allclose(h, fp * hp + fc * hc, rtol=1e-9, atol=1e-9 * np.max(np.abs(h)))
