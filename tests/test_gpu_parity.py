"""CUDA path against the FP64 oracle, through the C ABI.

Tolerances: |delta log L| <= 1e-3 per sample (the stated bound of the method); draws to
1e-12 relative (both sides evaluate the same Philox words in FP64); ESS and log Z to 1e-3
relative when computed from each side's own log L, and to 1e-12 when the reduction
alone is compared on identical inputs.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC
from oracle.events import make_event, make_proposal
from gpu_common import (LOGL_TOL, m, torch, to_fp32_data, gpu_context, set_metric, gpu_loglike,  # noqa: F401
                        compare_loglike, logl_bound)

pytestmark = pytest.mark.gpu


# --------------------------------------------------------------------------------- tiny event
@pytest.fixture(scope="module")
def tiny():
    w = workloads.tiny(n_samples=4096)
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    return w, spec, ev, th, prop


def test_draws_match_oracle(m, torch, tiny):
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, prop)
        for n, ctr0 in [(4096, 0), (1000, 123457)]:   # full and ragged batches
            P = len(prop["ids"])
            theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
            lq = torch.empty(n, dtype=torch.float64, device="cuda")
            lp = torch.empty(n, dtype=torch.float64, device="cuda")
            m.mbis_draw(ctx, spec.draw_seed, ctr0, n, theta, lq, lp)
            torch.cuda.synchronize()
            ref_th, ref_lq = oracle.draw(spec.draw_seed, ctr0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
            ref_lp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], ref_th)
            np.testing.assert_allclose(theta.cpu().numpy(), ref_th, rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(lq.cpu().numpy(), ref_lq, rtol=1e-12, atol=1e-12)
            g = lp.cpu().numpy()
            assert np.array_equal(np.isfinite(g), np.isfinite(ref_lp))
            np.testing.assert_allclose(g[np.isfinite(g)], ref_lp[np.isfinite(ref_lp)], rtol=1e-12, atol=1e-12)
    finally:
        m.mbis_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiny_loglike_matches_oracle(m, torch, tiny, precision):
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64 if precision == "fp64" else m.MIXED)
    try:
        set_metric(m, ctx, prop)
        theta, _ = oracle.draw(spec.draw_seed, 0, w.n_samples, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        logp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta)
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], theta, th))
        got = gpu_loglike(m, torch, ctx, theta)
        dmax = compare_loglike(got, ref, logp)
        if precision == "fp64":
            assert dmax < 1e-8
        # at the injection (zero noise): ln I0(rho^2) - rho^2 / 2
        t0 = np.array([[th[i]] for i in prop["ids"]])
        g0 = gpu_loglike(m, torch, ctx, t0)[0]
        assert abs(g0 - (oracle.log_i0([225.0])[0] - 112.5)) < (1e-8 if precision == "fp64" else LOGL_TOL)
    finally:
        m.mbis_destroy(ctx)


def test_cached_anchor_plan_gives_identical_likelihoods(m, torch, tiny):
    """The anchor plan depends only on the grid, the prior box and the tolerances, and the
    library keeps recent plans per process: a context whose plan comes from that cache
    evaluates every sample bit for bit as the context that built it.  A prior box no other
    test uses makes the first set-up build its plan afresh."""
    w, spec, ev, th, prop = tiny
    prop = dict(prop)
    prop["hi"] = np.array(prop["hi"], dtype=np.float64) * (1.0 + 1e-9)
    theta, _ = oracle.draw(spec.draw_seed, 0, 2048, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
    outs = []
    for _ in range(2):
        ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
        try:
            set_metric(m, ctx, prop)
            outs.append(gpu_loglike(m, torch, ctx, theta))
        finally:
            m.mbis_destroy(ctx)
    assert np.array_equal(outs[0], outs[1])


def test_reduce_matches_oracle(m, torch, tiny):
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, prop)
        n = w.n_samples
        P = len(prop["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq = torch.empty(n, dtype=torch.float64, device="cuda")
        lp = torch.empty(n, dtype=torch.float64, device="cuda")
        ll = torch.empty(n, dtype=torch.float64, device="cuda")
        wts = torch.empty(n, dtype=torch.float64, device="cuda")
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, ll)
        s = m.mbis_reduce(ctx, n, ll, lp, lq, wts)
        # oracle end to end on its own draws
        ref_th, ref_lq = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        ref_lp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], ref_th)
        ref_ll = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], ref_th, th))
        r = oracle.reduce(ref_ll, ref_lp, ref_lq, want_weights=True)
        assert abs(s["ess"] / r["ess"] - 1) < 1e-3
        assert abs(s["log_z"] - r["log_z"]) < 1e-3 * max(1.0, abs(r["log_z"]))
        assert s["n"] == n
        # the reduction alone on identical inputs
        d_ll = torch.tensor(ref_ll, device="cuda")
        d_lp = torch.tensor(ref_lp, device="cuda")
        d_lq = torch.tensor(ref_lq, device="cuda")
        s2 = m.mbis_reduce(ctx, n, d_ll, d_lp, d_lq, wts)
        assert abs(s2["ess"] / r["ess"] - 1) < 1e-12
        assert abs(s2["log_z"] - r["log_z"]) < 1e-12 * max(1.0, abs(r["log_z"]))
        np.testing.assert_allclose(wts.cpu().numpy(), r["weights"], rtol=1e-12, atol=1e-300)
    finally:
        m.mbis_destroy(ctx)


def test_reduce_edge_cases_and_accumulation(m, torch, tiny):
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        z = torch.zeros(0, dtype=torch.float64, device="cuda")
        s = m.mbis_reduce(ctx, 0, z, z, z)
        assert s["n"] == 0 and s["ess"] == 0 and s["all_zero"]
        n = 1000
        ninf = torch.full((n,), -math.inf, dtype=torch.float64, device="cuda")
        zero = torch.zeros(n, dtype=torch.float64, device="cuda")
        s = m.mbis_reduce(ctx, n, ninf, zero, zero)
        assert s["ess"] == 0 and s["log_z"] == -math.inf and s["all_zero"]
        # merging batches equals one batch
        rng = np.random.default_rng(2)
        ll = rng.normal(10, 3, 5000)
        lp = np.where(rng.uniform(size=5000) < 0.1, -np.inf, rng.normal(0, 1, 5000))
        lq = rng.normal(0, 1, 5000)
        T = lambda a: torch.tensor(a, device="cuda")
        whole = m.mbis_reduce(ctx, 5000, T(ll), T(lp), T(lq))
        m.mbis_reset_running(ctx)
        for a, b in [(0, 1234), (1234, 4000), (4000, 5000)]:
            part = m.mbis_reduce(ctx, b - a, T(ll[a:b]), T(lp[a:b]), T(lq[a:b]), accumulate=True)
        assert part["n"] == 5000
        assert abs(part["ess"] / whole["ess"] - 1) < 1e-12
        assert abs(part["log_z"] - whole["log_z"]) < 1e-12
    finally:
        m.mbis_destroy(ctx)


def test_unphysical_samples_get_minus_infinity(m, torch, tiny):
    w, spec, ev, th, prop = tiny
    for prec in (m.FP64, m.MIXED):
        ctx = gpu_context(m, ev, w, spec, th, prec)
        try:
            set_metric(m, ctx, prop)
            t = np.array([[th[MC], -1.0, th[MC], th[MC]], [th[Q], 1.2, 0.0, 1.2], [0.1, 0.1, 0.1, 1.5],
                          [0.0, 0.0, 0.0, 0.0]])
            got = gpu_loglike(m, torch, ctx, t)
            assert np.isfinite(got[0]) and np.all(got[1:] == -np.inf)
        finally:
            m.mbis_destroy(ctx)


# ------------------------------------------------------------------ BNS population, full grid
@pytest.fixture(scope="module")
def bns():
    w = workloads.bns_population(n_events=2, n_samples=1 << 20)
    spec = w.events[1]
    ev, th, _ = make_event(w, spec)
    to_fp32_data(ev)   # both sides see the complex64 / float32 data
    prop = make_proposal(ev, w, th)
    return w, spec, ev, th, prop


def test_split_launches_equal_the_full_launch(m, torch, bns):
    """A small launch (fewer tiles than the GPU has CTA slots) splits each tile's bins over
    several CTAs; the overlap is summed in fixed parts of the grid, so every sample's log L
    equals, bit for bit, the one from a launch too large to split, for ragged and tiny
    batches too."""
    w, spec, ev, th, prop = bns
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        n = 1 << 18
        theta = torch.empty((len(prop["ids"]), n), dtype=torch.float64, device="cuda")
        lq, lp, full = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, full)
        for k in (1 << 16, 5000, 129, 1):
            part = torch.empty(k, dtype=torch.float64, device="cuda")
            m.mbis_loglike(ctx, k, theta[:, :k].contiguous(), part)
            torch.cuda.synchronize()
            assert torch.equal(part, full[:k]), k
    finally:
        m.mbis_destroy(ctx)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bns_full_grid_matches_oracle(m, torch, bns, precision):
    w, spec, ev, th, prop = bns
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED if precision == "mixed" else m.FP64)
    try:
        set_metric(m, ctx, prop)
        n = 128
        theta, _ = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        theta[:, 0] = [th[i] for i in prop["ids"]]       # include the injection
        logp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta)
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], theta, th))
        got = gpu_loglike(m, torch, ctx, theta)
        compare_loglike(got, ref, logp)
    finally:
        m.mbis_destroy(ctx)


def test_bns_full_size_launch_sampled_outputs(m, torch, bns):
    """The benchmark's launch: 2^20 samples of one BNS event in one call; outputs at 96
    sampled indices against the oracle, and all outputs finite or -inf where invalid."""
    w, spec, ev, th, prop = bns
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        n = w.n_samples
        P = len(prop["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq = torch.empty(n, dtype=torch.float64, device="cuda")
        lp = torch.empty(n, dtype=torch.float64, device="cuda")
        ll = torch.empty(n, dtype=torch.float64, device="cuda")
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, ll)
        s = m.mbis_reduce(ctx, n, ll, lp, lq)
        torch.cuda.synchronize()
        llh = ll.cpu().numpy()
        assert not np.any(np.isnan(llh))
        idx = np.random.default_rng(7).choice(n, 96, replace=False)
        idx[0] = n - 1
        th_s = theta.cpu().numpy()[:, idx]
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], th_s, th))
        compare_loglike(llh[idx], ref, oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], th_s))
        assert s["ess"] > 100 and np.isfinite(s["log_z"])
    finally:
        m.mbis_destroy(ctx)


# ------------------------------------------------- BBH with full extrinsics, time marginalised
@pytest.fixture(scope="module")
def bbh():
    w = workloads.bbh_population(n_events=2, n_samples=1 << 12)
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    to_fp32_data(ev)
    prop = make_proposal(ev, w, th)
    return w, spec, ev, th, prop


def test_bbh_time_marginalised_fp64_matches_oracle(m, torch, bbh):
    w, spec, ev, th, prop = bbh
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, prop)
        n = 33   # ragged: one warp per sample
        theta, _ = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        theta[:, 0] = [th[i] for i in prop["ids"]]
        logp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta)
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], theta, th))
        got = gpu_loglike(m, torch, ctx, theta)
        assert compare_loglike(got, ref, logp) < 1e-6
    finally:
        m.mbis_destroy(ctx)


def test_weighted_moments_match_oracle(m, torch, tiny):
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, prop)
        n = 4097
        theta, lq = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        wts = np.random.default_rng(1).uniform(0, 1, n)
        wts[::5] = 0.0
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        mean, cov = m.mbis_weighted_moments(ctx, n, T(theta), T(wts))
        ref_mean, ref_cov = oracle.weighted_moments(prop["ids"], theta, wts, prop["mean"])
        np.testing.assert_allclose(mean, ref_mean, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(cov, ref_cov, rtol=1e-9, atol=1e-14 * np.max(np.abs(ref_cov)))
    finally:
        m.mbis_destroy(ctx)


def test_ess_loop_equals_manual_batches_and_refit_raises_efficiency(m, torch, tiny):
    """a7: with a fixed proposal the loop equals batches merged by hand; with refits it
    reaches the target ESS with fewer draws, and the evidence agrees within Monte-Carlo error."""
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        P, batch = len(prop["ids"]), 8192
        bufs = [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
               [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]
        s0, nd0, nu0 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=1 << 22,
                                         seed=spec.draw_seed, refine=0)
        assert nd0 == nu0 and s0["ess"] >= 300.0 and s0["n"] == nu0
        # the same batches by hand
        m.mbis_reset_running(ctx)
        theta, lq, lp, ll, _ = bufs
        for b in range(nu0 // batch):
            m.mbis_draw(ctx, spec.draw_seed, b * batch, batch, theta, lq, lp)
            m.mbis_loglike(ctx, batch, theta, ll)
            manual = m.mbis_reduce(ctx, batch, ll, lp, lq, None, True)
        assert abs(manual["ess"] / s0["ess"] - 1) < 1e-12 and abs(manual["log_z"] - s0["log_z"]) < 1e-12
        # refitted proposal
        set_metric(m, ctx, prop)
        s1, nd1, nu1 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=1 << 22,
                                         seed=spec.draw_seed, refine=2, refine_scale=1.2)
        assert s1["ess"] >= 300.0 and nu1 < nu0 and nd1 == nu1 + 2 * batch and s1["n"] == nu1
        assert s1["ess"] / nu1 > 3 * s0["ess"] / nu0
        # (no evidence comparison: on this event the Fisher proposal's weights are heavy-tailed
        # and its estimate of Z is biased low at this ESS -- the oracle shows the same)
        assert math.isfinite(s1["log_z"])
    finally:
        m.mbis_destroy(ctx)


def _oracle_ess_loop(ev, th, prop, seed, batch, target, max_samples, refine, refine_scale):
    """The ESS-target loop on the oracle (Eqs. 5-6; the refit of the proposal from weighted
    samples, Sec. III A): batch b draws the Philox counters [b batch, (b + 1) batch) from the
    current Gaussian; each of the first `refine` batches refits the mean and covariance from
    its normalised weights (when its own ESS is at least 2P + 1), with the width scale
    refine_scale, and does not enter the estimate; the later batches are reduced together
    until the ESS reaches the target.  Returns (summary, draws, draws in the estimate)."""
    ids = prop["ids"]
    P = len(ids)
    mean, chol, scale = np.array(prop["mean"], dtype=float), np.array(prop["chol"], dtype=float).reshape(P, P), \
        prop["scale"]
    refits, b, drawn = refine, 0, 0
    kept = ([], [], [])
    summary = None
    while drawn < max_samples:
        nb = min(batch, max_samples - drawn)
        theta, lq = oracle.draw(seed, b * batch, nb, ids, mean, chol, scale)
        lp = oracle.log_prior(ids, prop["lo"], prop["hi"], prop["flags"], theta)
        inside = np.isfinite(lp)
        ll = np.zeros(nb)
        ll[inside] = oracle.loglike_batch(ev, oracle.full_params(ids, theta[:, inside], th))
        drawn += nb
        b += 1
        if refits > 0:
            refits -= 1
            red = oracle.reduce(ll, lp, lq, want_weights=True)
            if red["ess"] >= 2 * P + 1:
                mean, cov = oracle.weighted_moments(ids, theta, red["weights"], mean)
                chol = np.linalg.cholesky(cov)
                scale = refine_scale if refine_scale > 0 else scale
            kept = ([], [], [])
            continue
        for k, x in enumerate((ll, lp, lq)):
            kept[k].append(x)
        summary = oracle.reduce(*(np.concatenate(x) for x in kept))
        if summary["ess"] >= target:
            break
    return summary, drawn, sum(len(x) for x in kept[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refitted_ess_loop_replayed_by_the_oracle(m, torch, tiny, precision):
    """a7 end to end: the loop with two refits on the device, and the same sequence of
    draws, likelihoods, weights, refits and merged estimates replayed by the oracle from its
    own arithmetic -- the same draw counts, and the final ESS and log Z to 1e-6 (FP64 path)
    or 1e-3 (mixed path) relative."""
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64 if precision == "fp64" else m.MIXED)
    try:
        set_metric(m, ctx, prop)
        P, batch, target = len(prop["ids"]), 4096, 400.0
        bufs = [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
               [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]
        got, nd, nu = m.mbis_run_to_ess(ctx, *bufs, ess_target=target, batch=batch, max_samples=64 * batch,
                                        seed=spec.draw_seed, refine=2, refine_scale=1.2)
        ref, nd_o, nu_o = _oracle_ess_loop(ev, th, prop, spec.draw_seed, batch, target, 64 * batch, 2, 1.2)
        tol = 1e-6 if precision == "fp64" else 1e-3
        print(f"  device: ESS {got['ess']:.3f} log Z {got['log_z']:.6f} drawn {nd} used {nu}; "
              f"oracle: ESS {ref['ess']:.3f} log Z {ref['log_z']:.6f} drawn {nd_o} used {nu_o}")
        assert (nd, nu) == (nd_o, nu_o) and nu > 0 and got["ess"] >= target
        assert abs(got["ess"] / ref["ess"] - 1) <= tol, (got["ess"], ref["ess"])
        assert abs(got["log_z"] - ref["log_z"]) <= tol * max(1.0, abs(ref["log_z"])), (got["log_z"], ref["log_z"])
    finally:
        m.mbis_destroy(ctx)


def test_ess_loop_pools_refit_batches_up_to_the_cap(m, torch, tiny):
    """a7 with refit_min_ess: a refit batch short of it pools with the next ones; with a
    floor that no pool reaches, each refit takes 16 batches; with no floor (0) the loop is
    the per-batch rule (one batch per refit)."""
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        P, batch = len(prop["ids"]), 4096
        bufs = [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
               [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]
        set_metric(m, ctx, prop)
        s0, nd0, nu0 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=1 << 22,
                                         seed=spec.draw_seed, refine=1, refine_scale=1.2)
        assert nd0 == nu0 + batch and s0["ess"] >= 300.0
        set_metric(m, ctx, prop)
        s1, nd1, nu1 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=1 << 22,
                                         seed=spec.draw_seed, refine=1, refine_scale=1.2, refit_min_ess=1e15)
        assert nd1 == nu1 + 16 * batch and s1["ess"] >= 300.0 and s1["n"] == nu1
        set_metric(m, ctx, prop)
        s2, nd2, nu2 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=1 << 22,
                                         seed=spec.draw_seed, refine=2, refine_scale=1.2, refit_min_ess=1e15)
        assert nd2 == nu2 + 32 * batch and s2["ess"] >= 300.0
        # the loop stops at max_samples while pooling, with nothing in the estimate
        set_metric(m, ctx, prop)
        s3, nd3, nu3 = m.mbis_run_to_ess(ctx, *bufs, ess_target=300.0, batch=batch, max_samples=5 * batch,
                                         seed=spec.draw_seed, refine=1, refit_min_ess=1e15)
        assert nd3 == 5 * batch and nu3 == 0 and s3["n"] == 0
    finally:
        m.mbis_destroy(ctx)


def test_pooled_refit_equals_the_weighted_moments_of_the_pooled_batches(m, torch, tiny):
    """a7 with refit_min_ess: two refit batches pooled (their moment sums rescaled to one
    weight scale) give the Gaussian that the weighted moments of the two batches taken as
    one draw give -- one reduction over both, one moment pass.  The seed is picked so that
    the two batches' largest log-weights differ by more than 1.5, which the rescaling must
    absorb."""
    w, spec, ev, th, prop = tiny
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, prop)
        P, batch = len(prop["ids"]), 1024
        theta = torch.empty((P, 2 * batch), dtype=torch.float64, device="cuda")
        lq, lp, ll, wt = (torch.empty(2 * batch, dtype=torch.float64, device="cuda") for _ in range(4))
        chosen = None
        for seed in range(spec.draw_seed, spec.draw_seed + 200):
            m.mbis_draw(ctx, seed, 0, 2 * batch, theta, lq, lp)
            m.mbis_loglike(ctx, 2 * batch, theta, ll)
            b0 = m.mbis_reduce(ctx, batch, ll[:batch], lp[:batch], lq[:batch])
            b1 = m.mbis_reduce(ctx, batch, ll[batch:], lp[batch:], lq[batch:])
            both = m.mbis_reduce(ctx, 2 * batch, ll, lp, lq, wt)
            floor = 0.5 * (b0["ess"] + both["ess"])
            if abs(b0["max_logw"] - b1["max_logw"]) > 1.5 and both["ess"] > b0["ess"] + 2 and floor > 2 * P + 1:
                chosen = seed, floor
                break
        assert chosen is not None, "no seed with two batches of different weight scale"
        seed, floor = chosen
        mean_r, cov_r = m.mbis_weighted_moments(ctx, 2 * batch, theta, wt)
        chol_r = np.linalg.cholesky(cov_r)
        # the loop: the first batch falls short of the floor and pools with the second
        bufs = [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
               [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]
        _, nd, nu = m.mbis_run_to_ess(ctx, *bufs, ess_target=1e30, batch=batch, max_samples=2 * batch, seed=seed,
                                      refine=1, refine_scale=1.3, refit_min_ess=floor)
        assert nd == 2 * batch and nu == 0
        mean_g, chol_g, scale_g = m.mbis_get_proposal(ctx, P)
        assert scale_g == 1.3
        sd = np.sqrt(np.diag(cov_r))
        assert np.max(np.abs(mean_g - mean_r) / sd) < 1e-12
        assert np.max(np.abs(chol_g - chol_r) / sd[:, None]) < 1e-12
        # a floor that the first batch meets on its own refits from that batch alone
        if b0["ess"] >= 2 * P + 1.5:
            th1, lq1, lp1, ll1, w1 = bufs
            set_metric(m, ctx, prop)
            m.mbis_draw(ctx, seed, 0, batch, th1, lq1, lp1)
            m.mbis_loglike(ctx, batch, th1, ll1)
            m.mbis_reduce(ctx, batch, ll1, lp1, lq1, w1)
            mean_1, cov_1 = m.mbis_weighted_moments(ctx, batch, th1, w1)
            m.mbis_run_to_ess(ctx, *bufs, ess_target=1e30, batch=batch, max_samples=batch, seed=seed, refine=1,
                              refine_scale=1.3, refit_min_ess=2 * P + 1.5)
            mean_g1, chol_g1, _ = m.mbis_get_proposal(ctx, P)
            sd1 = np.sqrt(np.diag(cov_1))
            assert np.max(np.abs(mean_g1 - mean_1) / sd1) < 1e-12
            assert np.max(np.abs(chol_g1 - np.linalg.cholesky(cov_1)) / sd1[:, None]) < 1e-12
    finally:
        m.mbis_destroy(ctx)


def test_bbh_time_marginalised_tensor_core_matches_oracle(m, torch, bbh):
    """The tcgen05 time-shift contraction (split TF32, FP32 accumulation in TMEM) against
    the oracle; 300 samples = one full CTA of 256 and a ragged second one."""
    w, spec, ev, th, prop = bbh
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        n = 300
        theta, _ = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        theta[:, 0] = [th[i] for i in prop["ids"]]
        logp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta)
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], theta, th))
        got = gpu_loglike(m, torch, ctx, theta)
        inside = np.isfinite(logp)
        print(f"tensor-core time marginalisation: max |delta log L| = {np.abs(got - ref)[inside].max():.2e}, "
              f"mean signed {np.mean((got - ref)[inside]):+.2e}")
        compare_loglike(got, ref, logp)
    finally:
        m.mbis_destroy(ctx)


def test_time_kernel_sample_order_leaves_results_unchanged(m, torch, bbh):
    """Launches of 4096 or more samples hand them to the CTAs in order of their live
    K-blocks (a permutation computed on the device); every sample's log L equals, bit for
    bit, the one from launches too small to be reordered."""
    w, spec, ev, th, prop = bbh
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        n, P = 3 * 4096 + 77, len(prop["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq, lp, full = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, full)
        for a in range(0, n, 2000):
            k = min(2000, n - a)
            part = torch.empty(k, dtype=torch.float64, device="cuda")
            m.mbis_loglike(ctx, k, theta[:, a:a + k].contiguous(), part)
            torch.cuda.synchronize()
            assert torch.equal(part, full[a:a + k]), a
    finally:
        m.mbis_destroy(ctx)


def test_bbh_full_size_tensor_core_launch_sampled_outputs(m, torch, bbh):
    """The benchmark's BBH launch: 2^18 samples of one event (11 parameters, 128 shifts) in
    one call of the tcgen05 kernel; 200 sampled outputs (in and out of the prior box)
    against the oracle, and no NaN anywhere."""
    w, spec, ev, th, prop = bbh
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        n, P = 1 << 18, len(prop["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq = torch.empty(n, dtype=torch.float64, device="cuda")
        lp = torch.empty(n, dtype=torch.float64, device="cuda")
        ll = torch.empty(n, dtype=torch.float64, device="cuda")
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, ll)
        torch.cuda.synchronize()
        llh = ll.cpu().numpy()
        assert not np.any(np.isnan(llh))
        idx = np.random.default_rng(11).choice(n, 200, replace=False)
        idx[0] = n - 1
        th_s = theta.cpu().numpy()[:, idx]
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], th_s, th))
        logp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], th_s)
        # every sample with a physical parameter set, in or out of the prior box, is held to
        # the same per-sample bound as the samples inside it
        phys = np.isfinite(ref)
        d = np.abs(llh[idx] - ref)[phys]
        print(f"full-size tensor-core launch: max |delta log L| = {d.max():.2e} over {phys.sum()} samples")
        compare_loglike(llh[idx], ref, logp)
        assert np.all(d <= logl_bound(ref[phys]))
    finally:
        m.mbis_destroy(ctx)
