"""Pins of the oracle's random numbers, proposal draws, priors and weight reduction.

Each test ties the oracle to something other than itself: published known-answer
vectors, scipy's independent distributions and special functions, closed-form
Gaussian integrals, and the paper's special case that a proposal equal to the target
gives ESS = N (App. A, discussion of Eq. 6).
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats, integrate

import oracle
from oracle import MC, Q, CHI1, CHI2, TC, RA, DEC, PSI, IOTA, DL, PHIC

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        assert list(oracle.philox4x32_10(w[:4], w[4:6])) == w[6:]


def test_box_muller_normals_are_standard_normal():
    # identity proposal: theta = z exactly
    n, P = 200_000, 4
    theta, logq = oracle.draw(12345, 0, n, [MC, Q, CHI1, CHI2], np.zeros(P), np.eye(P), 1.0)
    z = theta.ravel()
    assert abs(z.mean()) < 5 * 1 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # components are uncorrelated
    c = np.corrcoef(theta)
    assert np.max(np.abs(c - np.eye(P))) < 5 / math.sqrt(n)
    # log g equals the standard normal log density
    ref = stats.multivariate_normal(np.zeros(P), np.eye(P)).logpdf(theta.T)
    np.testing.assert_allclose(logq, ref, rtol=0, atol=1e-10)


def test_draw_counter_addressing():
    # sample i of a batch starting at ctr0 equals sample 0 of a batch starting at ctr0 + i
    P = 5
    mean = np.array([1.2, 1.3, 0.01, -0.02, 0.0])
    L = np.tril(np.random.default_rng(0).uniform(0.1, 0.3, (P, P))) + np.eye(P)
    a, la = oracle.draw(99, 1000, 64, [MC, Q, CHI1, CHI2, TC], mean, L, 1.5)
    b, lb = oracle.draw(99, 1037, 1, [MC, Q, CHI1, CHI2, TC], mean, L, 1.5)
    np.testing.assert_array_equal(a[:, 37], b[:, 0])
    assert la[37] == lb[0]
    # P = 11 uses three Philox blocks; the first four normals match the P = 4 draw
    c, _ = oracle.draw(99, 1000, 8, list(range(4)), np.zeros(4), np.eye(4), 1.0)
    d, _ = oracle.draw(99, 1000, 8, [MC, Q, CHI1, CHI2, 4, 5, 6, 7, 8, 9, 10], np.zeros(11), np.eye(11), 1.0)
    # RA (slot 4) and psi/phi_c wrap; compare unwrapped slots only
    np.testing.assert_array_equal(c, d[:4])


def test_draw_moments_and_density():
    rng = np.random.default_rng(1)
    P = 5
    A = rng.normal(size=(P, P))
    cov = A @ A.T + P * np.eye(P)
    L = np.linalg.cholesky(cov)
    mean = rng.normal(size=P) + np.array([10, 2, 0, 0, 0])
    s = 1.5
    n = 100_000
    theta, logq = oracle.draw(7, 0, n, [MC, Q, CHI1, CHI2, TC], mean, L, s)
    assert np.all(np.abs(theta.mean(axis=1) - mean) < 6 * s * np.sqrt(np.diag(cov) / n))
    emp = np.cov(theta)
    np.testing.assert_allclose(emp, s * s * cov, rtol=0, atol=0.05 * s * s * np.max(np.diag(cov)))
    ref = stats.multivariate_normal(mean, s * s * cov).logpdf(theta.T)
    np.testing.assert_allclose(logq, ref, rtol=0, atol=1e-9)


def test_angles_wrap_into_their_periods():
    P = 3
    theta, _ = oracle.draw(5, 0, 20000, [RA, PSI, PHIC], np.array([6.0, 3.0, 0.1]), 2.0 * np.eye(P), 1.0)
    assert theta[0].min() >= 0 and theta[0].max() < 2 * math.pi
    assert theta[1].min() >= 0 and theta[1].max() < math.pi
    assert theta[2].min() >= 0 and theta[2].max() < 2 * math.pi


def _prior_1d_integral(pid, lo, hi, flags=0, n=200001):
    xs = np.linspace(lo, hi, n)
    lp = oracle.log_prior([pid], [lo], [hi], flags, xs[None, :])
    return integrate.trapezoid(np.exp(lp), xs)


@pytest.mark.parametrize("pid,lo,hi", [(MC, 1.0, 1.4), (CHI1, -0.99, 0.99), (TC, -0.01, 0.01),
                                        (DEC, -math.pi / 2, math.pi / 2), (DEC, -0.3, 0.7),
                                        (IOTA, 0.0, math.pi), (DL, 10.0, 1000.0)])
def test_prior_normalises(pid, lo, hi):
    assert abs(_prior_1d_integral(pid, lo, hi) - 1.0) < 1e-6


def test_periodic_priors_and_outside_box():
    for pid, period in [(RA, 2 * math.pi), (PSI, math.pi), (PHIC, 2 * math.pi)]:
        lp = oracle.log_prior([pid], [0.0], [period], 0, np.array([[0.5]]))
        assert abs(lp[0] + math.log(period)) < 1e-14
    assert oracle.log_prior([MC], [1.0], [2.0], 0, np.array([[2.5]]))[0] == -np.inf
    assert oracle.log_prior([DEC], [-1.0], [1.0], 0, np.array([[1.2]]))[0] == -np.inf


def test_component_mass_prior_normalises_and_has_the_jacobian():
    mc_lo, mc_hi, q_lo, q_hi = 1.1, 1.3, 1.0, 2.5
    # the normalisation against scipy's adaptive quadrature of the Jacobian
    ref, _ = integrate.dblquad(lambda q, mc: oracle.mass_jacobian(mc, q), mc_lo, mc_hi, q_lo, q_hi,
                               epsabs=0, epsrel=1e-12)
    assert abs(oracle.mass_prior_volume(mc_lo, mc_hi, q_lo, q_hi) / ref - 1) < 1e-10
    # a density flat in (m1, m2): its ratio at two points equals the Jacobian ratio
    th = np.array([[1.15, 1.25], [1.1, 2.2]])
    lp = oracle.log_prior([MC, Q], [mc_lo, q_lo], [mc_hi, q_hi], oracle.PRIOR_M1M2, th)
    assert abs((lp[0] - lp[1]) - math.log(oracle.mass_jacobian(1.15, 1.1) / oracle.mass_jacobian(1.25, 2.2))) < 1e-12
    # and it integrates to one over the box
    g = 401
    mcs, qs = np.linspace(mc_lo, mc_hi, g), np.linspace(q_lo, q_hi, g)
    MM, QQ = np.meshgrid(mcs, qs, indexing="ij")
    lp = oracle.log_prior([MC, Q], [mc_lo, q_lo], [mc_hi, q_hi], oracle.PRIOR_M1M2, np.stack([MM.ravel(), QQ.ravel()]))
    tot = integrate.trapezoid(integrate.trapezoid(np.exp(lp).reshape(g, g), qs, axis=1), mcs)
    assert abs(tot - 1) < 1e-5


# ---------------------------------------------------------------------------------------
# Eqs. 5-6: weights, Kish ESS and evidence


def test_equal_weights_give_ess_n():
    n = 1000
    r = oracle.reduce(np.full(n, 3.0), np.full(n, -1.0), np.full(n, 0.5), want_weights=True)
    assert abs(r["ess"] - n) < 1e-9
    assert abs(r["log_z"] - 1.5) < 1e-13
    np.testing.assert_allclose(r["weights"], 1.0 / n, rtol=1e-14)


def test_single_nonzero_weight_gives_ess_one():
    n = 50
    ll = np.full(n, -np.inf)
    ll[17] = 2.0
    r = oracle.reduce(ll, np.zeros(n), np.zeros(n))
    assert abs(r["ess"] - 1.0) < 1e-15
    assert abs(r["log_z"] - (2.0 - math.log(n))) < 1e-13


def test_all_zero_weights():
    r = oracle.reduce(np.full(10, -np.inf), np.zeros(10), np.zeros(10))
    assert r["ess"] == 0.0 and r["log_z"] == -np.inf


def test_reduce_against_scipy_logsumexp():
    rng = np.random.default_rng(3)
    n = 100_000
    ll, lp, lq = rng.normal(50, 4, n), rng.normal(-3, 1, n), rng.normal(-2, 1, n)
    lp[::97] = -np.inf
    r = oracle.reduce(ll, lp, lq, want_weights=True)
    lw = ll + lp - lq
    assert abs(r["log_z"] - (special.logsumexp(lw) - math.log(n))) < 1e-10
    ess_ref = math.exp(2 * special.logsumexp(lw) - special.logsumexp(2 * lw))
    assert abs(r["ess"] / ess_ref - 1) < 1e-10
    assert abs(r["weights"].sum() - 1) < 1e-12


def test_weighted_moments_against_numpy_and_wrap():
    rng = np.random.default_rng(4)
    n, ids = 5000, [MC, Q, CHI1, RA]
    theta = np.stack([rng.normal(1.2, 1e-4, n), rng.normal(1.5, 0.1, n), rng.normal(0, 0.02, n),
                      np.mod(rng.normal(0.05, 0.1, n), 2 * math.pi)])     # RA straddles 0 = 2 pi
    w = rng.uniform(0, 1, n)
    w[::7] = 0.0
    ref = np.array([1.2, 1.5, 0.0, 6.2])
    mean, cov = oracle.weighted_moments(ids, theta, w, ref)
    lin = theta.copy()
    lin[3] = np.where(lin[3] > math.pi, lin[3] - 2 * math.pi, lin[3])    # unwrapped reference copy
    mu = np.average(lin, axis=1, weights=w)
    ref_cov = np.cov(lin, aweights=w, bias=True)
    np.testing.assert_allclose(mean[:3], mu[:3], rtol=1e-12, atol=1e-14)
    assert abs(((mean[3] - mu[3] + math.pi) % (2 * math.pi)) - math.pi) < 1e-12
    np.testing.assert_allclose(cov, ref_cov, rtol=1e-9, atol=1e-18)


def test_proposal_equal_to_target_gives_ess_n_and_closed_form_evidence():
    """App. A (after Eq. 6): a proposal equal to the posterior makes every weight equal."""
    rng = np.random.default_rng(11)
    P = 4
    A = rng.normal(size=(P, P))
    gamma = A @ A.T + 2 * np.eye(P)              # target precision (a Fisher matrix)
    cov = np.linalg.inv(gamma)
    L = np.linalg.cholesky(cov)
    mu = np.array([20.0, 2.0, 0.1, -0.1])
    n = 4096
    theta, logq = oracle.draw(21, 0, n, [MC, Q, CHI1, CHI2], mu, L, 1.0)
    c = 7.25
    d = theta - mu[:, None]
    loglike = -0.5 * np.einsum("in,ij,jn->n", d, gamma, d) + c
    half = 50 * np.sqrt(np.diag(cov))            # flat prior box far wider than the target
    lo, hi = mu - half, mu + half
    logp = oracle.log_prior([MC, Q, CHI1, CHI2], lo, hi, 0, theta)
    r = oracle.reduce(loglike, logp, logq)
    assert abs(r["ess"] - n) < 1e-9 * n
    logv = np.sum(np.log(hi - lo))
    ref = c + 0.5 * P * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(gamma)[1] - logv
    assert abs(r["log_z"] - ref) < 1e-9
