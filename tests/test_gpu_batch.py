"""Uneven multi-event batch against the single-event path and the FP64 oracle, through the
C ABI.

One step of a batch draws every event's samples, evaluates all of them in one persistent
likelihood launch over a shared work list of (event, 128-sample tile) items, and reduces
each event to its summary, replayed from a CUDA graph.  A tile runs the same per-sample
arithmetic in the persistent launch as in the single-event launch, so the log L of every
sample must be bitwise equal to mbis_loglike's; against the oracle the bound is
|delta log L| <= 1e-3 per sample.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, make_proposal
from gpu_common import LOGL_TOL, m, torch, gpu_context, set_metric, compare_loglike  # noqa: F401

pytestmark = pytest.mark.gpu

ORACLE_SAMPLES = 64   # oracle log L per event, spread over the event's samples


def build(ws, mod, n_samples):
    """Oracle events and proposals; GPU contexts (mixed precision) with the proposals set."""
    out = []
    for w, n in zip(ws, n_samples):
        w.n_samples = n
        spec = w.events[0]
        ev, th, _ = make_event(w, spec)
        prop = make_proposal(ev, w, th)
        ctx = gpu_context(mod, ev, w, spec, th, mod.MIXED)
        set_metric(mod, ctx, prop)
        out.append(dict(w=w, spec=spec, ev=ev, th=th, prop=prop, ctx=ctx))
    return out


def check_step(mod, torch, b, evs, step):
    """Summaries of one batch step against the single-event entry points, and a sample of
    each event's log L against the oracle."""
    sums = mod.mbis_batch_step(b, step, len(evs))
    for i, e in enumerate(evs):
        n, P = e["w"].n_samples, len(e["prop"]["ids"])
        theta_b, ll_b = mod.mbis_batch_copy_out(b, i, P, n)
        # the same draws as the single-event call at counter step * n
        th = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq = torch.empty(n, dtype=torch.float64, device="cuda")
        lp = torch.empty(n, dtype=torch.float64, device="cuda")
        ll = torch.empty(n, dtype=torch.float64, device="cuda")
        mod.mbis_draw(e["ctx"], e["spec"].draw_seed, step * n, n, th, lq, lp)
        mod.mbis_loglike(e["ctx"], n, th, ll)
        ref = mod.mbis_reduce(e["ctx"], n, ll, lp, lq, None, 0)
        torch.cuda.synchronize()
        assert np.array_equal(theta_b, th.cpu().numpy()), e["w"].name
        assert np.array_equal(ll_b, ll.cpu().numpy(), equal_nan=True), e["w"].name
        for k in ("ess", "log_z", "max_logw", "s1", "s2"):
            assert sums[i][k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), (e["w"].name, k)
        assert sums[i]["n"] == n
        # oracle on an evenly spread sample of the event's draws
        idx = np.unique(np.linspace(0, n - 1, min(n, ORACLE_SAMPLES)).astype(np.int64))
        sub = theta_b[:, idx]
        logp = oracle.log_prior(e["prop"]["ids"], e["prop"]["lo"], e["prop"]["hi"], e["prop"]["flags"], sub)
        want = oracle.loglike_batch(e["ev"], oracle.full_params(e["prop"]["ids"], sub, e["th"]))
        compare_loglike(ll_b[idx], want, logp)
    return sums


@pytest.fixture(scope="module")
def small(m):
    # six events of both families, 2 and 3 detectors, 1,969 to 64,257 bins, sample counts
    # that are not multiples of the 128-sample tile (and one single partial tile)
    ws = workloads.uneven_batch()[:6]
    evs = build(ws, m, [1000, 3000, 129, 4096, 777, 2500])
    yield evs
    for e in evs:
        m.mbis_destroy(e["ctx"])


def test_batch_steps_equal_single_event_path_and_oracle(m, torch, small):
    evs = small
    b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                            [e["spec"].draw_seed for e in evs])
    try:
        s0 = check_step(m, torch, b, evs, 0)
        check_step(m, torch, b, evs, 1)          # the graph replays with new Philox counters
        s0_again = m.mbis_batch_step(b, 0, len(evs))
        assert s0_again == s0                    # replays are deterministic
        # a proposal moved between steps is picked up by the next step (re-captured graph)
        p = evs[1]["prop"]
        m.mbis_set_proposal(evs[1]["ctx"], p["mean"] * (1 + 1e-6), p["chol"] * 0.5, p["scale"])
        try:
            check_step(m, torch, b, evs, 2)
        finally:
            m.mbis_set_proposal(evs[1]["ctx"], p["mean"], p["chol"], p["scale"])
    finally:
        m.mbis_batch_destroy(b)


def oracle_summary(e, theta_b, step=0):
    """The oracle's reduction of its own log L on event e's draws of a batch step (samples
    outside the prior have zero weight and are not evaluated)."""
    n, prop, spec = e["w"].n_samples, e["prop"], e["spec"]
    ref_th, ref_lq = oracle.draw(spec.draw_seed, step * n, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
    np.testing.assert_allclose(theta_b, ref_th, rtol=1e-12, atol=1e-13)
    ref_lp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], ref_th)
    inside = np.isfinite(ref_lp)
    ref_ll = np.zeros(n)
    ref_ll[inside] = oracle.loglike_batch(e["ev"], oracle.full_params(prop["ids"], ref_th[:, inside], e["th"]))
    return oracle.reduce(ref_ll, ref_lp, ref_lq), ref_ll, ref_lp


def test_batch_summaries_match_the_oracle(m, torch, small):
    """Configuration 4 end to end: each event's ESS and log Z from one batch step against
    the oracle's reduction of its own log L on every draw of that event (relative ESS and
    absolute log Z to 1e-3)."""
    evs = small
    b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                            [e["spec"].draw_seed for e in evs])
    try:
        sums = m.mbis_batch_step(b, 1, len(evs))
        for i, e in enumerate(evs):
            theta_b, ll_b = m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)
            ref, ref_ll, ref_lp = oracle_summary(e, theta_b, step=1)
            compare_loglike(ll_b, ref_ll, ref_lp)
            print(f"  {e['w'].name}: ESS {sums[i]['ess']:.3f} (oracle {ref['ess']:.3f}), "
                  f"log Z {sums[i]['log_z']:.5f} (oracle {ref['log_z']:.5f})")
            assert sums[i]["n"] == ref["n"]
            assert abs(sums[i]["ess"] / ref["ess"] - 1) <= 1e-3
            assert abs(sums[i]["log_z"] - ref["log_z"]) <= 1e-3
    finally:
        m.mbis_batch_destroy(b)


def test_batch_with_fp64_block_entry_events(m, torch):
    """Events whose t_c phase term exceeds 2^16 turns enter their anchor blocks in FP64; a
    batch holding both kinds runs one persistent launch for each.  Both equal the
    single-event path bit for bit and the oracle within the bounds."""
    import copy
    ws = workloads.uneven_batch()[:3]
    ws = [copy.deepcopy(w) for w in ws]
    ws[1].events[0].params["tc"] = 200.0    # 200 s x 512-1024 Hz > 2^16 turns
    evs = build(ws, m, [700, 900, 300])
    try:
        kinds = [m.mbis_get_info(e["ctx"])["ff_phase"] for e in evs]
        assert kinds == [1, 0, 1], kinds
        b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                                [e["spec"].draw_seed for e in evs])
        try:
            sums = check_step(m, torch, b, evs, 0)
            for i, e in enumerate(evs):
                theta_b, _ = m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)
                ref, _, _ = oracle_summary(e, theta_b)
                assert abs(sums[i]["ess"] / ref["ess"] - 1) <= 1e-3
                assert abs(sums[i]["log_z"] - ref["log_z"]) <= 1e-3
        finally:
            m.mbis_batch_destroy(b)
    finally:
        for e in evs:
            m.mbis_destroy(e["ctx"])


def test_batch_autotune_keeps_results(m, torch, small):
    evs = small
    b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                            [e["spec"].draw_seed for e in evs])
    try:
        before = m.mbis_batch_step(b, 3, len(evs))
        grid, ms = m.mbis_batch_autotune(b)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        tile, grid2 = m.mbis_batch_shape(b)
        assert grid2 == grid and tile in (64, 128, 256)
        assert grid % sms == 0 and 1 <= grid // sms <= {64: 14, 128: 7, 256: 3}[tile]
        assert ms > 0.0
        after = m.mbis_batch_step(b, 3, len(evs))
        assert after == before
        # the persistent launch alone on a caller stream recomputes the same log L
        lls = [m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)[1] for i, e in enumerate(evs)]
        s = torch.cuda.Stream()
        m.mbis_batch_loglike(b, s)
        s.synchronize()
        for i, e in enumerate(evs):
            again = m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)[1]
            assert np.array_equal(again, lls[i])
    finally:
        m.mbis_batch_destroy(b)


def test_batch_rejects_unsupported_contexts(m, torch, small):
    evs = small
    with pytest.raises(m.MbisError):
        m.mbis_batch_create([evs[0]["ctx"]], [0], [1])
    w = workloads.tiny()
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        set_metric(m, ctx, make_proposal(ev, w, th))
        with pytest.raises(m.MbisError):
            m.mbis_batch_create([evs[0]["ctx"], ctx], [128, 128], [1, 2])
    finally:
        m.mbis_destroy(ctx)


@pytest.mark.parametrize("tile,ctas", [(64, 14), (256, 3), (64, 5)])
def test_batch_tile_shapes_keep_results(m, torch, small, tile, ctas):
    """Every tile shape the autotuner tries gives the same log L and summaries, bit for bit:
    a sample's arithmetic does not depend on how many samples share its CTA."""
    evs = small
    b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                            [e["spec"].draw_seed for e in evs])
    try:
        ref = m.mbis_batch_step(b, 4, len(evs))
        lls = [m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)[1] for i, e in enumerate(evs)]
        m.mbis_batch_set_shape(b, tile, ctas)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert m.mbis_batch_shape(b) == (tile, sms * ctas)
        assert m.mbis_batch_step(b, 4, len(evs)) == ref
        for i, e in enumerate(evs):
            assert np.array_equal(m.mbis_batch_copy_out(b, i, len(e["prop"]["ids"]), e["w"].n_samples)[1], lls[i])
        with pytest.raises(m.MbisError):
            m.mbis_batch_set_shape(b, 96, 2)
    finally:
        m.mbis_batch_destroy(b)


def test_batch_full_size_events(m, torch):
    """Eight events of the uneven population at their full sample counts (2^14 to 2^20,
    2 million samples in all) and full grids (1,969 to 64,257 bins), in the autotuned
    persistent launch: every sample bitwise equal to the single-event path, 64 per event
    against the oracle."""
    ws = workloads.uneven_batch()[:8]
    evs = build(ws, m, [w.n_samples for w in ws])
    try:
        b = m.mbis_batch_create([e["ctx"] for e in evs], [e["w"].n_samples for e in evs],
                                [e["spec"].draw_seed for e in evs])
        try:
            m.mbis_batch_autotune(b)
            sums = check_step(m, torch, b, evs, 0)
            assert all(s["ess"] >= 1.0 for s in sums)
        finally:
            m.mbis_batch_destroy(b)
    finally:
        for e in evs:
            m.mbis_destroy(e["ctx"])
