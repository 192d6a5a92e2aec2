"""Relative binning through the C ABI: the device likelihood against the oracle's on the
same samples, fiducial and bins (|delta log L| <= 1e-3), its state rules, and its
closeness to the exact likelihood with bins from mbis_rb_edges."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, make_proposal
from gpu_common import LOGL_TOL, m, torch, gpu_context, set_metric  # noqa: F401

pytestmark = pytest.mark.gpu


def draws(prop, n, seed):
    theta, _ = oracle.draw(seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
    lp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta)
    return theta, np.isfinite(lp)


def test_tiny_event_with_isco_cuts_matches_the_oracle(m, torch):
    """Phase marginalised, 1969 bins of which ~240 lie below the ISCO: bins of 16 grid
    points, so that every sample's cut falls inside a bin."""
    w = workloads.tiny()
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        edges = np.array(list(range(0, w.n_bins, 16)) + [w.n_bins], dtype=np.int32)
        theta, inside = draws(prop, 2048, 5)
        with pytest.raises(m.MbisError):
            m.mbis_rb_loglike(ctx, 4, torch.tensor(theta[:, :4], device="cuda"),
                              torch.empty(4, dtype=torch.float64, device="cuda"))
        m.mbis_rb_setup(ctx, th, edges)
        ll = torch.empty(theta.shape[1], dtype=torch.float64, device="cuda")
        m.mbis_rb_loglike(ctx, theta.shape[1], torch.tensor(theta, device="cuda"), ll)
        got = ll.cpu().numpy()
        want = oracle.rb_loglike_batch(ev, th, edges, oracle.full_params(prop["ids"], theta, th))
        d = np.abs(got[inside] - want[inside])
        assert d.max() <= LOGL_TOL, d.max()
        # a new metric drops the set-up
        set_metric(m, ctx, prop)
        with pytest.raises(m.MbisError):
            m.mbis_rb_loglike(ctx, theta.shape[1], torch.tensor(theta, device="cuda"), ll)
        print(f"tiny: max |delta log L| vs oracle {d.max():.2e}")
    finally:
        m.mbis_destroy(ctx)


def test_bns_event_matches_the_oracle_and_stays_close_to_the_exact_likelihood(m, torch):
    """Phase and distance marginalised BNS event on 20-512 Hz at 1/128 Hz (62,977 bins);
    bins from mbis_rb_edges (5 proposal sigmas, 0.05 rad per bin)."""
    w = workloads.scaled(workloads.bns_population(n_events=1), f_hi=512.0)
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        edges = m.mbis_rb_edges(ctx, th, 5.0, 0.05)
        assert edges[0] == 0 and edges[-1] == w.n_bins and np.all(np.diff(edges) > 0)
        assert len(m.mbis_rb_edges(ctx, th, 5.0, 0.2)) < len(edges)
        m.mbis_rb_setup(ctx, th, edges)
        theta, inside = draws(prop, 1 << 16, 9)
        n = theta.shape[1]
        th_d = torch.tensor(theta, device="cuda")
        rb, ex = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2))
        m.mbis_rb_loglike(ctx, n, th_d, rb)
        m.mbis_loglike(ctx, n, th_d, ex)
        rb, ex = rb.cpu().numpy(), ex.cpu().numpy()
        sub = np.flatnonzero(inside)[::1024][:48]
        want = oracle.rb_loglike_batch(ev, th, edges, oracle.full_params(prop["ids"], theta[:, sub], th))
        d = np.abs(rb[sub] - want)
        assert d.max() <= LOGL_TOL, d.max()
        # against the exact likelihood: the samples that carry the posterior
        lw = ex[inside] - ex[inside].max()
        heavy = lw > -10.0
        err = np.abs(rb[inside] - ex[inside])[heavy]
        assert np.median(err) < 1e-2 and err.max() < 0.1
        print(f"BNS: {len(edges) - 1} coarse bins for {w.n_bins}; vs oracle {d.max():.2e}; vs exact on "
              f"{heavy.sum()} posterior samples: median {np.median(err):.1e}, max {err.max():.1e}")
    finally:
        m.mbis_destroy(ctx)
