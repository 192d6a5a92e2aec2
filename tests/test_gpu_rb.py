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


def test_ess_loop_runs_on_the_relative_binning_likelihood(m, torch):
    """mbis_rb_use routes mbis_loglike (and so the ESS loop) through relative binning: the
    same draws give the same log L as mbis_rb_loglike, bit for bit; without refits the loop
    draws the same samples as the exact run, so ESS and log Z agree to the parity tolerance;
    a proposal refit keeps the set-up, a new metric drops it and restores the exact path."""
    w = workloads.scaled(workloads.bns_population(n_events=1), f_hi=256.0)
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        with pytest.raises(m.MbisError):
            m.mbis_rb_use(ctx, True)
        m.mbis_rb_setup(ctx, th, m.mbis_rb_edges(ctx, th, 5.0, 0.05))
        theta, _ = draws(prop, 1 << 14, 11)
        n = theta.shape[1]
        th_d = torch.tensor(theta, device="cuda")
        rb, via = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2))
        m.mbis_rb_loglike(ctx, n, th_d, rb)
        m.mbis_rb_use(ctx, True)
        m.mbis_loglike(ctx, n, th_d, via)
        torch.cuda.synchronize()
        assert torch.equal(rb, via)

        P, batch = len(prop["ids"]), 1 << 14
        bufs = [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
               [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]
        runs = {}
        for use in (True, False):
            m.mbis_rb_use(ctx, use)
            runs[use] = m.mbis_run_to_ess(ctx, *bufs, 2000.0, batch, 1 << 18, 77, refine=0)
        (s_rb, nd_rb, _), (s_ex, nd_ex, _) = runs[True], runs[False]
        assert nd_rb == nd_ex
        assert abs(s_rb["ess"] / s_ex["ess"] - 1) < 1e-3
        assert abs(s_rb["log_z"] - s_ex["log_z"]) < 1e-3 * max(1.0, abs(s_ex["log_z"]))

        # a refit keeps the set-up
        m.mbis_set_proposal(ctx, prop["mean"], prop["chol"], prop["scale"] * 0.9)
        m.mbis_rb_use(ctx, True)
        m.mbis_loglike(ctx, n, th_d, via)
        # a new metric drops it: mbis_loglike is the exact likelihood again
        set_metric(m, ctx, prop)
        with pytest.raises(m.MbisError):
            m.mbis_rb_loglike(ctx, n, th_d, rb)
        ex = torch.empty(n, dtype=torch.float64, device="cuda")
        m.mbis_loglike(ctx, n, th_d, ex)
        torch.cuda.synchronize()
        assert not torch.equal(ex, via)
        print(f"ESS loop on relative binning: ESS {s_rb['ess']:.1f} vs {s_ex['ess']:.1f}, "
              f"log Z {s_rb['log_z']:.5f} vs {s_ex['log_z']:.5f}, {nd_rb} drawn")
    finally:
        m.mbis_destroy(ctx)
