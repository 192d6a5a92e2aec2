"""Pins of the oracle's credible level (the P-P test of Sec. III A): order statistics,
symmetry, ties, and the exact posterior of a conjugate Gaussian model."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def test_equal_weights_give_the_empirical_cdf():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 1000))
    ref = np.array([0.3, -1.2, 2.0])
    got = oracle.credible_levels(x, np.ones(1000), ref)
    want = [(x[p] < ref[p]).mean() for p in range(3)]
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_mirror_symmetric_samples_put_the_centre_at_one_half_and_ties_count_half():
    x = np.concatenate([np.linspace(-3, 3, 101), -np.linspace(-3, 3, 101)])[None, :]  # includes 0 twice
    w = np.concatenate([np.linspace(1, 2, 101), np.linspace(1, 2, 101)])
    assert oracle.credible_levels(x, w, [0.0])[0] == pytest.approx(0.5, abs=1e-15)
    # all mass at the reference: one half
    assert oracle.credible_levels(np.zeros((1, 5)), np.ones(5), [0.0])[0] == 0.5
    # weights of any positive scale; non-positive weights are skipped
    a = oracle.credible_levels(x, w, [0.7])[0]
    b = oracle.credible_levels(x, 1e-200 * w, [0.7])[0]
    assert a == pytest.approx(b, rel=1e-14)


def test_importance_weighted_level_matches_the_exact_gaussian_posterior():
    """Prior N(0, 1) on a mean, one datum y ~ N(mu, s^2): the posterior is N(y/(1+s^2),
    s^2/(1+s^2)).  Samples from the prior weighted by the likelihood give the posterior CDF
    at any reference within Monte-Carlo error."""
    rng = np.random.default_rng(7)
    y, s2 = 0.8, 0.5
    mu = rng.normal(size=400000)
    w = np.exp(-0.5 * (y - mu) ** 2 / s2)
    post_m, post_v = y / (1 + s2), s2 / (1 + s2)
    for ref in (-0.2, 0.5, 0.9):
        got = oracle.credible_levels(mu[None, :], w, [ref])[0]
        assert got == pytest.approx(stats.norm.cdf(ref, post_m, math.sqrt(post_v)), abs=4e-3)


def test_levels_of_the_truth_are_uniform_over_a_simulated_population():
    """Draw truths from the prior, data from the model, and weighted prior samples: the
    levels of the truths pass a KS test against U(0, 1)."""
    rng = np.random.default_rng(11)
    levels = []
    mu = rng.normal(size=20000)
    for _ in range(300):
        truth = rng.normal()
        y = truth + math.sqrt(0.5) * rng.normal()
        w = np.exp(-0.5 * (y - mu) ** 2 / 0.5)
        levels.append(oracle.credible_levels(mu[None, :], w, [truth])[0])
    assert stats.kstest(levels, "uniform").pvalue > 0.01
