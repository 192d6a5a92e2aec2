"""The library's Gaussian proposal from a Fisher matrix (mbis_proposal_from_fisher, host
arithmetic of Sec. II A: Schur complement of the marginalised slots, prior-width term,
inverse, Cholesky factor, prior box) against the test side's own recipe on the same
matrix.  No device is used: the library call is pure host code."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, marginalised_slots, proposal_fisher, proposal_from_fisher


@pytest.fixture(scope="module")
def m():
    import paper_2410_05190_gb300 as mod
    return mod


def _cases():
    tiny = workloads.tiny(n_samples=16)
    bns = workloads.scaled(workloads.bns_population(n_events=2, n_samples=16), f_hi=256.0)
    bbh = workloads.bbh_population(n_events=2, n_samples=16)
    return [("tiny", tiny, tiny.events[0]), ("bns", bns, bns.events[1]), ("bbh", bbh, bbh.events[0])]


@pytest.mark.parametrize("name,w,spec", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_proposal_from_fisher_matches_the_recipe(m, name, w, spec):
    ev, th, _ = make_event(w, spec)
    G = proposal_fisher(ev, w, th)
    extra = marginalised_slots(w.marg)
    ref = proposal_from_fisher(G, w.sampled, th, w.scale, w.box_sigmas, w.chi_max, w.dmin, w.dmax, w.prior_flags)
    got = m.mbis_proposal_from_fisher(list(w.sampled), extra, G, th, scale=w.scale, box_sigmas=w.box_sigmas,
                                      chi_max=w.chi_max, dmin=w.dmin, dmax=w.dmax, prior_flags=w.prior_flags)
    assert np.array_equal(got["ids"], ref["ids"])
    np.testing.assert_array_equal(got["mean"], ref["mean"])
    # the factor reproduces the covariance of the recipe to rounding of a P <= 11 inverse
    cg, cr = got["chol"] @ got["chol"].T, ref["chol"] @ ref["chol"].T
    np.testing.assert_allclose(cg, cr, rtol=1e-9, atol=1e-12 * np.abs(cr).max())
    np.testing.assert_allclose(got["chol"], ref["chol"], rtol=1e-8, atol=1e-10 * np.abs(ref["chol"]).max())
    assert np.all(np.triu(got["chol"], 1) == 0) and np.all(np.diag(got["chol"]) > 0)
    np.testing.assert_allclose(got["lo"], ref["lo"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(got["hi"], ref["hi"], rtol=1e-10, atol=1e-14)


def test_schur_complement_equals_the_conditional_precision(m):
    """For a Gaussian with precision G the marginal over the last slots has precision
    A - B C^-1 B^T; with a prior-width-free slot set (Mc, t_c) the proposal covariance is
    then the leading block of G^-1 exactly."""
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, 4))
    G = X.T @ X + 4 * np.eye(4)
    th = np.zeros(11)
    th[workloads.MC], th[workloads.TC] = 10.0, 0.0
    got = m.mbis_proposal_from_fisher([workloads.MC, workloads.TC], [workloads.PHIC, workloads.DL], G, th,
                                      scale=1.0)
    cov = got["chol"] @ got["chol"].T
    np.testing.assert_allclose(cov, np.linalg.inv(G)[:2, :2], rtol=1e-12)
    # the box is +-10 proposal sigmas about the trigger
    np.testing.assert_allclose(got["hi"] - th[[workloads.MC, workloads.TC]], 10 * np.sqrt(np.diag(cov)), rtol=1e-12)


def test_prior_width_term_and_periodic_boxes(m):
    """A slot the data do not constrain at all gets the variance of a uniform distribution
    over its prior range (width^2 / 12); angle slots get their full range as the box."""
    ids = [workloads.CHI1, workloads.RA, workloads.PSI, workloads.Q]
    G = np.zeros((4, 4))
    th = np.zeros(11)
    th[workloads.Q] = 1.5
    got = m.mbis_proposal_from_fisher(ids, [], G, th, scale=1.0, chi_max=0.9)
    var = np.diag(got["chol"] @ got["chol"].T)
    np.testing.assert_allclose(var, [1.8 ** 2 / 12, (2 * math.pi) ** 2 / 12, math.pi ** 2 / 12, 4.0 / 12], rtol=1e-13)
    np.testing.assert_allclose(got["lo"], [-0.9, 0.0, 0.0, 1.0])
    np.testing.assert_allclose(got["hi"], [0.9, 2 * math.pi, math.pi, 1.5 + 10 * math.sqrt(4.0 / 12)], rtol=1e-13)


def test_bad_inputs_are_rejected(m):
    th = np.zeros(11)
    with pytest.raises(m.MbisError) as e:      # not positive definite (Mc has no prior width)
        m.mbis_proposal_from_fisher([workloads.MC], [], np.zeros((1, 1)), th)
    assert e.value.status == m.MBIS_E_INVALID
    with pytest.raises(m.MbisError):           # a slot both sampled and marginalised
        m.mbis_proposal_from_fisher([workloads.MC], [workloads.MC], np.eye(2), th)
    with pytest.raises(m.MbisError):           # non-finite entry
        m.mbis_proposal_from_fisher([workloads.MC], [], np.array([[np.nan]]), th)
    with pytest.raises(m.MbisError):           # bad option: a sampled spin with chi_max = 1
        m.mbis_proposal_from_fisher([workloads.CHI1], [], np.eye(1), th, chi_max=1.0)
    with pytest.raises(m.MbisError):           # bad option: a sampled distance with dmin = 0
        m.mbis_proposal_from_fisher([workloads.DL], [], np.eye(1), th, dmin=0.0)
    with pytest.raises(m.MbisError):           # bad option: scale 0
        m.mbis_proposal_from_fisher([workloads.MC], [], np.eye(1), th, scale=0.0)


def test_unsampled_spin_and_distance_bounds_are_not_checked(m):
    """A non-spinning proposal over (Mc, q) needs no spin or distance range: chi_max = 0 and
    an empty distance range are accepted and change nothing."""
    th = np.zeros(11)
    th[workloads.MC], th[workloads.Q] = 20.0, 1.2
    G = np.array([[4.0e4, 1.0e2], [1.0e2, 9.0]])
    a = m.mbis_proposal_from_fisher([workloads.MC, workloads.Q], [], G, th, chi_max=0.0, dmin=0.0, dmax=0.0)
    b = m.mbis_proposal_from_fisher([workloads.MC, workloads.Q], [], G, th, chi_max=0.9)
    for k in ("mean", "chol", "lo", "hi"):
        np.testing.assert_array_equal(a[k], b[k])
