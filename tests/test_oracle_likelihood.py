"""Pins of the oracle's likelihood (Eqs. 1-3) and its marginalisations (Sec. III).

The marginalised likelihoods are tied to brute-force averages of the unmarginalised
likelihood over phi_c, d_L and t_c; log I0 to scipy and to quadrature; the injection to
log L = SNR^2 / 2; the noise to its defining second moments; the Fisher matrix to the
closed forms of its amplitude and phase entries.
"""
import math

import numpy as np
import pytest
from scipy import special, integrate

import oracle
import workloads
from workloads import MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC
from oracle.events import make_event


def small_workload(marg, detectors=("H1", "L1"), f_hi=128.0, df=0.25, snr=15.0, noise_seed=None):
    spec = workloads.EventSpec(m1=20.0, m2=14.0,
                               params=dict(chi1=0.2, chi2=-0.1, ra=2.0, dec=-0.4, psi=1.1, iota=0.9, tc=0.0, phic=0.7),
                               gmst=0.3, snr=snr, noise_seed=noise_seed, draw_seed=1)
    w = workloads.Workload("small", list(detectors), 20.0, f_hi, df, [MC, Q, CHI1, CHI2], marg, 64, "fp64", "c128",
                           1.0, 0, 0.99, [spec])
    return w, spec


def test_log_i0_against_scipy_and_quadrature():
    xs = np.concatenate([np.linspace(0, 5, 11), [29.9, 30.0, 30.1, 100.0, 700.0, 2500.0, 1e4]])
    ref = np.log(special.i0e(xs)) + xs
    got = oracle.log_i0(xs)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)
    for x in [0.5, 12.0, 45.0, 900.0]:
        n = 4096
        phi = 2 * math.pi * np.arange(n) / n
        quad = x + math.log(np.mean(np.exp(x * (np.cos(phi) - 1))))
        assert abs(oracle.log_i0([x])[0] - quad) < 1e-12 * max(1, x)


def test_zero_noise_injection_gives_half_snr_squared():
    w, spec = small_workload(0)
    ev, th, dl = make_event(w, spec)
    assert abs(oracle.optimal_snr2(ev, th) - 225.0) < 1e-9
    assert abs(oracle.loglike(ev, th) - 112.5) < 1e-9
    evp = ev.with_marg(oracle.MARG_PHASE)
    assert abs(oracle.loglike(evp, th) - (oracle.log_i0([225.0])[0] - 112.5)) < 1e-9
    assert abs(oracle.loglike(evp, th) - 108.8735) < 1e-3


def test_phase_marginal_equals_brute_force_average_over_phi_c():
    w, spec = small_workload(0, noise_seed=77)
    ev, th, _ = make_event(w, spec)
    evp = ev.with_marg(oracle.MARG_PHASE)
    n = 512
    for dmc in [0.0, 0.002, -0.01]:
        p = th.copy()
        p[MC] *= 1 + dmc
        rows = np.tile(p, (n, 1))
        rows[:, PHIC] = 2 * math.pi * np.arange(n) / n
        ll = oracle.loglike_batch(ev, rows)
        brute = special.logsumexp(ll) - math.log(n)
        assert abs(oracle.loglike(evp, p) - brute) < 1e-9


def test_distance_marginal_equals_brute_force_and_scipy_quad():
    w, spec = small_workload(0, noise_seed=78)
    ev, th, dl_true = make_event(w, spec)
    dmin, dmax = 10.0, 1000.0
    evd = ev.with_marg(oracle.MARG_PHASE | oracle.MARG_DISTANCE, dmin=dmin, dmax=dmax)
    evp = ev.with_marg(oracle.MARG_PHASE)
    for dmc in [0.0, 0.003]:
        p = th.copy()
        p[MC] *= 1 + dmc
        got = oracle.loglike(evd, p)
        # (1) quadrature of the phase-marginalised likelihood evaluated at each distance
        ds = np.linspace(dmin, dmax, 40001)
        rows = np.tile(p, (len(ds), 1))
        rows[:, DL] = ds
        ll = oracle.loglike_batch(evp, rows) + np.log(3 * ds ** 2 / (dmax ** 3 - dmin ** 3))
        m = ll.max()
        brute = m + math.log(integrate.simpson(np.exp(ll - m), x=ds))
        assert abs(got - brute) < 1e-6
        # (2) scipy adaptive quadrature of the same integrand from (Z1, H1)
        q = p.copy()
        q[DL], q[PHIC] = 1.0, 0.0
        z1, h1 = oracle.overlaps(ev, q)
        g = lambda d: math.log(3 * d * d / (dmax ** 3 - dmin ** 3)) + oracle.log_i0([abs(z1) / d])[0] - h1 / (2 * d * d)
        peak = max(dmin, min(dmax, h1 / abs(z1)))
        ref, _ = integrate.quad(lambda d: math.exp(g(d) - m), dmin, dmax, points=[peak], epsabs=0, epsrel=1e-12,
                                limit=500)
        assert abs(oracle.distance_marginal(abs(z1), h1, dmin, dmax) - (m + math.log(ref))) < 1e-10


def test_time_marginal_equals_brute_force_over_shifted_t_c():
    w, spec = small_workload(0, detectors=("H1", "L1", "V1"), noise_seed=79)
    ev, th, _ = make_event(w, spec)
    J, dt = 128, 1e-4
    evt = ev.with_marg(oracle.MARG_TIME, n_tshift=J, dt_shift=dt)
    for dtc in [0.0, 3.3e-4]:
        p = th.copy()
        p[TC] += dtc
        rows = np.tile(p, (J, 1))
        rows[:, TC] = p[TC] + (np.arange(J) - J // 2) * dt
        ll = oracle.loglike_batch(ev, rows)
        brute = special.logsumexp(ll) - math.log(J)
        assert abs(oracle.loglike(evt, p) - brute) < 1e-8


def test_cauchy_schwarz_and_parameter_independent_norm():
    w, spec = small_workload(0, noise_seed=80)
    ev, th, _ = make_event(w, spec)
    dd = 0.0
    for d in range(ev.n_det):
        s = ev.strain[d, :, 0] + 1j * ev.strain[d, :, 1]
        dd += 4 * w.df * np.sum(np.abs(s) ** 2 / ev.psd[d])
    rng = np.random.default_rng(0)
    for _ in range(10):
        p = th.copy()
        p[MC] *= 1 + rng.normal(0, 0.01)
        p[CHI1] = rng.uniform(-0.5, 0.5)
        z, hh = oracle.overlaps(ev, p)
        assert abs(z) <= math.sqrt(dd * hh) * (1 + 1e-12)
        q = p.copy()
        q[TC] += 0.01
        q[PHIC] += 2.0
        assert abs(oracle.overlaps(ev, q)[1] / hh - 1) < 1e-13


def test_noise_has_the_stated_second_moments():
    nb = 256
    f = 20 + 0.25 * np.arange(nb)
    psd = oracle.psd_aligo(f)[None, :]
    v, x, y = workloads.network(["H1"])
    ev = oracle.OracleEvent(20.0, 0.25, nb, psd, v, x, y)
    th = np.array([20.0, 1.4, 0.1, 0.0, 1.0, 0.2, 0.3, 0.5, 100.0, 0.0, 0.0])
    h = ev.with_marg(0)
    _, hh = oracle.overlaps(h, th)     # strain is zero here; hh = (h|h)
    nn, nh = [], []
    for seed in range(400):
        n = oracle.make_strain(ev, th, seed, True) - oracle.make_strain(ev, th, 0, False)
        ev.set_strain(n)
        nn.append(np.sum(4 * 0.25 * (n[0, :, 0] ** 2 + n[0, :, 1] ** 2) / psd[0]) / nb)
        z, _ = oracle.overlaps(ev, th)
        nh.append(z.real)
    assert abs(np.mean(nn) - 2.0) < 5 * math.sqrt(4.0 / nb / 400)
    assert abs(np.var(nh) / hh - 1) < 5 * math.sqrt(2 / 400)


def test_fisher_amplitude_and_phase_entries_have_closed_forms():
    w, spec = small_workload(0)
    ev, th, dl = make_event(w, spec)
    rho2 = oracle.optimal_snr2(ev, th)
    ids = [DL, PHIC, TC]
    G = oracle.fisher(ev.with_marg(0), th, ids, [1e-4 * dl, 1e-5, 1e-7])
    assert abs(G[0, 0] * dl * dl / rho2 - 1) < 1e-7       # dh/d(ln d) = -h
    assert abs(G[1, 1] / rho2 - 1) < 1e-8                 # dh/dphi_c = i h
    assert abs(G[0, 1]) < 1e-8 * math.sqrt(G[0, 0] * G[1, 1])
    # dh/dt_c = -2 pi i f h: Gamma_tt = sum 4 df (2 pi f)^2 |h|^2 / S
    f = ev.freqs()
    tt = 0.0
    for d in range(ev.n_det):
        h = oracle.detector_strain(ev, d, f, th)
        tt += np.sum(4 * w.df * (2 * math.pi * f) ** 2 * np.abs(h) ** 2 / ev.psd[d])
    assert abs(G[2, 2] / tt - 1) < 1e-6
