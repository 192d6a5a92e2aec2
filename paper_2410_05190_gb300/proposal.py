"""Gaussian proposal in the Fisher metric at a trigger (Sec. II A), from the library's own
FP64 Fisher matrix (mbis_fisher).

The proposal of the method is a multivariate Gaussian whose covariance is the inverse
of the likelihood metric at the trigger point.  Slots that the likelihood marginalises
(phi_c under phase marginalisation, d_L under distance marginalisation) are projected
out of the metric by a Schur complement.  Directions the data barely constrain (mass
ratio, spins, angles) get a weak Gaussian term of the prior's width (variance width^2 / 12,
that of a uniform distribution over the prior) so the proposal stays inside the prior.
The prior box is box_sigmas proposal standard deviations around the trigger for Mc, q and
t_c, and the physical range for the other slots.
"""
from __future__ import annotations

import math

import numpy as np

MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC = range(11)
MARG_PHASE, MARG_DISTANCE = 1, 2

# central-difference steps of the Fisher matrix (relative for Mc and d_L, absolute otherwise)
FISHER_STEPS = {MC: 1e-6, Q: 1e-6, CHI1: 1e-5, CHI2: 1e-5, RA: 1e-6, DEC: 1e-6, PSI: 1e-6, IOTA: 1e-6,
                DL: 1e-5, TC: 1e-7, PHIC: 1e-6}


def fisher_proposal(m, ctx, theta, sampled, marg, scale=1.5, box_sigmas=10.0, chi_max=0.99, dmin=10.0,
                    dmax=1000.0, prior_flags=0):
    """Proposal dict (ids, mean, chol, scale, lo, hi, flags) for mbis_set_metric.

    m: the binding module; ctx: a context of the event (its PSD, detectors and grid are
    used); theta: the 11 slot values of the trigger; sampled: the slots drawn."""
    sampled = list(sampled)
    extra = ([PHIC] if marg & MARG_PHASE else []) + ([DL] if marg & MARG_DISTANCE else [])
    ids = sampled + extra
    steps = np.array([FISHER_STEPS[i] * (theta[i] if i in (MC, DL) else 1.0) for i in ids])
    G = m.mbis_fisher(ctx, theta, ids, steps)
    P = len(sampled)
    if extra:
        A, B, Cm = G[:P, :P], G[:P, P:], G[P:, P:]
        G = A - B @ np.linalg.solve(Cm, B.T)
    else:
        G = G[:P, :P]
    width = {Q: 2.0, CHI1: 2 * chi_max, CHI2: 2 * chi_max, RA: 2 * math.pi, DEC: math.pi, PSI: math.pi,
             IOTA: math.pi, PHIC: 2 * math.pi, DL: dmax - dmin}
    for p, i in enumerate(sampled):
        if i in width:
            G[p, p] += 12.0 / width[i] ** 2
    cov = np.linalg.inv(G)
    cov = 0.5 * (cov + cov.T)
    L = np.linalg.cholesky(cov)
    sig = np.sqrt(np.diag(cov)) * scale
    mean = np.array([theta[i] for i in sampled])
    lo, hi = np.zeros(P), np.zeros(P)
    for p, i in enumerate(sampled):
        if i in (CHI1, CHI2):
            lo[p], hi[p] = -chi_max, chi_max
        elif i == Q:
            lo[p], hi[p] = max(1.0, theta[i] - box_sigmas * sig[p]), theta[i] + box_sigmas * sig[p]
        elif i in (MC, TC):
            lo[p], hi[p] = theta[i] - box_sigmas * sig[p], theta[i] + box_sigmas * sig[p]
        elif i in (RA, PHIC):
            lo[p], hi[p] = 0.0, 2 * math.pi
        elif i == PSI:
            lo[p], hi[p] = 0.0, math.pi
        elif i == DEC:
            lo[p], hi[p] = -math.pi / 2, math.pi / 2
        elif i == IOTA:
            lo[p], hi[p] = 0.0, math.pi
        elif i == DL:
            lo[p], hi[p] = dmin, dmax
    return dict(ids=np.array(sampled, dtype=np.int32), mean=mean, chol=L, scale=scale, lo=lo, hi=hi,
                flags=prior_flags)
