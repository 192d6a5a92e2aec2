"""P-P self-consistency of the posteriors (Sec. III A).

Over sources drawn from the prior, injected into noise and analysed with the same prior, the
credible level of each true parameter -- the posterior weight below it -- is uniform on
[0, 1].  The paper checks this per parameter with a Kolmogorov-Smirnov test and combines the
p-values.  The levels are computed on the device (mbis_credible_levels) from each event's
importance-weighted samples; this module runs a population through the tiled proposal and
holds the two statistics.  Every per-sample step runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np


def ks_pvalue(levels):
    """p-value of the one-sample Kolmogorov-Smirnov test of the levels against U(0, 1)."""
    from scipy import stats
    return float(stats.kstest(np.asarray(levels, dtype=np.float64), "uniform").pvalue)


def combined_pvalue(pvalues):
    """Fisher's combination of independent p-values: -2 sum ln p ~ chi^2 with 2k degrees."""
    from scipy import stats
    p = np.clip(np.asarray(pvalues, dtype=np.float64), 1e-300, 1.0)
    return float(stats.chi2.sf(-2.0 * np.log(p).sum(), 2 * len(p)))


def levels(m, torch, n, theta, weights, truth):
    """Credible levels of truth [P] under the weighted samples theta [P][n] (device)."""
    out = torch.empty(len(truth), dtype=torch.float64, device="cuda")
    m.mbis_credible_levels(n, theta, weights, truth, out)
    return out.cpu().numpy()


class TiledAnalysis:
    """Per-event analysis with a tiled proposal of the two-parameter space: a likelihood
    context over the space's physical (Mc, q) for the event's data, the template
    likelihoods, the mixture, draws, likelihoods, weights and the levels of the truth."""

    def __init__(self, m, torch, tiling, phys_templates, mc_range, q_range, n_samples):
        self.m, self.torch, self.t = m, torch, tiling
        self.n = n_samples
        self.T = phys_templates.shape[1]
        self.phys = torch.tensor(np.ascontiguousarray(phys_templates), dtype=torch.float64, device="cuda")
        self.mc_range, self.q_range = mc_range, q_range
        n = n_samples
        dev = dict(dtype=torch.float64, device="cuda")
        self.theta, self.coords = torch.empty((2, n), **dev), torch.empty((2, n), **dev)
        self.lq, self.lp, self.ll, self.w = (torch.empty(n, **dev) for _ in range(4))
        self.ll_t = torch.empty(self.T, **dev)

    def run(self, strain, psd, dets, f_lo, df, fixed, gmst, truth_xq, seed):
        """Returns (levels of x and q, summary) for one event's data."""
        m = self.m
        ctx = m.mbis_create(strain, psd, dets, f_lo, df, fixed, gmst=gmst, precision=m.MIXED, marg=m.MARG_PHASE)
        try:
            m.mbis_set_metric(ctx, np.array([0, 1], dtype=np.int32), np.array([sum(self.mc_range) / 2, 2.0]),
                              np.diag([0.1, 0.1]), 1.0, np.array([self.mc_range[0], self.q_range[0]]),
                              np.array([self.mc_range[1], self.q_range[1]]), 0)
            m.mbis_loglike(ctx, self.T, self.phys, self.ll_t)
            m.mbis_tiling_set_loglike(self.t, self.ll_t)
            m.mbis_tiling_draw(self.t, seed, 0, self.n, self.theta, self.lq, self.lp, coords=self.coords)
            m.mbis_loglike(ctx, self.n, self.theta, self.ll)
            s = m.mbis_reduce(ctx, self.n, self.ll, self.lp, self.lq, self.w)
            lv = levels(m, self.torch, self.n, self.coords, self.w, truth_xq)
        finally:
            m.mbis_destroy(ctx)
        return lv, s
