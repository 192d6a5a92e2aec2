"""Synthetic events and proposals built with the FP64 oracle (test infrastructure).

Every array produced here comes from the oracle (or from the seeded recipes in
``workloads``), never from the CUDA path, so it can serve as input to both sides of a
parity comparison, as the source of expected values, and as the input of the timed CPU
baseline.
"""
import math

import numpy as np

import oracle
import workloads
from workloads import MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC


def true_params(spec: workloads.EventSpec, dl=1.0):
    m1, m2 = spec.m1, spec.m2
    mc = (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2
    p = np.zeros(11)
    p[MC], p[Q] = mc, m1 / m2
    for k, v in spec.params.items():
        p[workloads.PARAM_NAMES.index(k)] = v
    p[DL] = dl
    return p


def make_event(w: workloads.Workload, spec: workloads.EventSpec, n_bins=None, noise=True):
    """Oracle event with injected signal (+ noise when the spec has a seed) at the
    requested network SNR.  Returns (event, theta_true, d_L)."""
    nb = w.n_bins if n_bins is None else n_bins
    f = w.f_lo + w.df * np.arange(nb)
    psd1 = oracle.psd_aligo(f)
    psd = np.tile(psd1, (w.n_det, 1))
    v, x, y = workloads.network(w.detectors)
    ev = oracle.OracleEvent(w.f_lo, w.df, nb, psd, v, x, y, gmst=spec.gmst, marg=w.marg, n_tshift=w.n_tshift,
                            dt_shift=w.dt_shift, dmin=w.dmin, dmax=w.dmax)
    th = true_params(spec, dl=1.0)
    rho1 = math.sqrt(oracle.optimal_snr2(ev, th))
    th[DL] = rho1 / spec.snr
    add_noise = noise and spec.noise_seed is not None
    ev.set_strain(oracle.make_strain(ev, th, spec.noise_seed or 0, add_noise))
    return ev, th, th[DL]


FISHER_STEPS = {MC: 1e-6, Q: 1e-6, CHI1: 1e-5, CHI2: 1e-5, RA: 1e-6, DEC: 1e-6, PSI: 1e-6, IOTA: 1e-6,
                DL: 1e-5, TC: 1e-7, PHIC: 1e-6}


def marginalised_slots(marg):
    """Slots the likelihood marginalises, in the order the proposal projects them out."""
    extra = []
    if marg & workloads.MARG_PHASE:
        extra.append(PHIC)
    if marg & workloads.MARG_DISTANCE:
        extra.append(DL)
    return extra


def fisher_steps(ids, th):
    return np.array([FISHER_STEPS[i] * (th[i] if i in (MC, DL) else 1.0) for i in ids])


def proposal_from_fisher(G, sampled, th, scale, box_sigmas, chi_max, dmin, dmax, prior_flags=0):
    """Gaussian proposal from the Fisher matrix G over sampled + marginalised slots (the
    last len(G) - len(sampled) rows): the marginalised slots are projected out by Schur
    complement; a weak Gaussian term of the prior width keeps directions the data cannot
    measure inside the prior; the prior box of Mc, q, t_c is +-box_sigmas proposal sigmas."""
    sampled = list(sampled)
    P = len(sampled)
    G = np.array(G, dtype=np.float64)
    if len(G) > P:
        A, B, Cm = G[:P, :P], G[:P, P:], G[P:, P:]
        G = A - B @ np.linalg.solve(Cm, B.T)
    else:
        G = G[:P, :P].copy()
    width = {Q: 2.0, CHI1: 2 * chi_max, CHI2: 2 * chi_max, RA: 2 * math.pi, DEC: math.pi, PSI: math.pi,
             IOTA: math.pi, PHIC: 2 * math.pi, DL: dmax - dmin}
    for p, i in enumerate(sampled):
        if i in width:
            G[p, p] += 12.0 / width[i] ** 2
    cov = np.linalg.inv(G)
    cov = 0.5 * (cov + cov.T)
    L = np.linalg.cholesky(cov)
    sig = np.sqrt(np.diag(cov)) * scale
    mean = np.array([th[i] for i in sampled])
    lo, hi = np.zeros(P), np.zeros(P)
    for p, i in enumerate(sampled):
        if i in (CHI1, CHI2):
            lo[p], hi[p] = -chi_max, chi_max
        elif i == Q:
            lo[p], hi[p] = max(1.0, th[i] - box_sigmas * sig[p]), th[i] + box_sigmas * sig[p]
        elif i in (MC, TC):
            lo[p], hi[p] = th[i] - box_sigmas * sig[p], th[i] + box_sigmas * sig[p]
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


def proposal_fisher(ev, w: workloads.Workload, th):
    """The oracle's Fisher matrix over the sampled slots followed by the marginalised ones."""
    ids = list(w.sampled) + marginalised_slots(w.marg)
    return oracle.fisher(ev.with_marg(0), th, ids, fisher_steps(ids, th))


def make_proposal(ev, w: workloads.Workload, th):
    """Gaussian proposal in the Fisher metric at the trigger (here the injection)."""
    G = proposal_fisher(ev, w, th)
    return proposal_from_fisher(G, w.sampled, th, w.scale, w.box_sigmas, w.chi_max, w.dmin, w.dmax, w.prior_flags)
