"""The P-P test is only meaningful when the injected sources follow the analysis prior
(Sec. III A).  The P-P populations draw (m1, m2) flat in a square and keep the pairs whose
(Mc, q) fall in the analysis box; that is the flat-(m1, m2) prior on the box only if the
square holds the whole box.  Checked here on the box's boundary, and the drawn truths
against the box and against the prior's Mc and q marginals."""
import numpy as np
import pytest
from scipy import integrate, stats

import workloads
from workloads import MC, Q, TC

CASES = [(workloads.bns_pp_population, workloads.PP_BOX, workloads.PP_MASS_SQUARE, 0.05),
         (workloads.bbh_pp_population, workloads.PP_BOX_BBH, workloads.PP_MASS_SQUARE_BBH, 0.8)]


def _masses(mc, q):
    m2 = mc * (1 + q) ** 0.2 / q ** 0.6
    return q * m2, m2


def _jacobian(mc, q):
    # |d(m1, m2) / d(Mc, q)| of m1 = q m2, m2 = Mc (1+q)^(1/5) q^(-3/5)
    return mc * (1 + q) ** 0.4 / q ** 1.2


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mass_square_holds_the_analysis_box(case):
    _, box, (lo, hi), _ = CASES[case]
    t = np.linspace(0.0, 1.0, 2001)
    (a, b), (c, d) = box[MC], box[Q]
    edges = [(a + (b - a) * t, np.full_like(t, c)), (a + (b - a) * t, np.full_like(t, d)),
             (np.full_like(t, a), c + (d - c) * t), (np.full_like(t, b), c + (d - c) * t)]
    for mc, q in edges:
        m1, m2 = _masses(mc, q)
        assert m2.min() >= lo and m1.max() <= hi


@pytest.mark.parametrize("case", range(len(CASES)))
def test_truths_follow_the_flat_mass_prior_on_the_box(case):
    make, box, _, chi_max = CASES[case]
    w = make(n_events=1500)
    mc = np.array([(e.m1 * e.m2) ** 0.6 / (e.m1 + e.m2) ** 0.2 for e in w.events])
    q = np.array([e.m1 / e.m2 for e in w.events])
    tc = np.array([e.params["tc"] for e in w.events])
    chi = np.array([[e.params["chi1"], e.params["chi2"]] for e in w.events])
    assert (mc >= box[MC][0]).all() and (mc <= box[MC][1]).all()
    assert (q >= box[Q][0]).all() and (q <= box[Q][1]).all()
    assert (tc >= box[TC][0]).all() and (tc <= box[TC][1]).all()
    assert np.abs(chi).max() <= chi_max and w.chi_max == chi_max
    (a, b), (c, d) = box[MC], box[Q]
    z = integrate.dblquad(lambda qq, m: _jacobian(m, qq), a, b, c, d)[0]

    def cdf_mc(x):
        return np.array([integrate.dblquad(lambda qq, m: _jacobian(m, qq), a, v, c, d)[0] / z for v in np.atleast_1d(x)])

    def cdf_q(x):
        return np.array([integrate.dblquad(lambda qq, m: _jacobian(m, qq), a, b, c, v)[0] / z for v in np.atleast_1d(x)])

    grid_mc, grid_q = np.linspace(a, b, 201), np.linspace(c, d, 201)
    fm, fq = cdf_mc(grid_mc), cdf_q(grid_q)
    assert stats.kstest(mc, lambda x: np.interp(x, grid_mc, fm)).pvalue > 1e-3
    assert stats.kstest(q, lambda x: np.interp(x, grid_q, fq)).pvalue > 1e-3
