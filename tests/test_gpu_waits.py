"""Failure detection without a GPU fault: a device wait on an mbarrier that nothing
completes gives up after its limit and reports MBIS_E_TIMEOUT; the context stays usable
(a likelihood evaluated right after matches the oracle)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, make_proposal
from gpu_common import m, torch, gpu_context, set_metric, gpu_loglike, compare_loglike  # noqa: F401

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_survives(m, torch):
    status, waited = m.mbis_debug_wait_timeout(2_000_000)   # 2 ms
    assert status == m.MBIS_E_TIMEOUT
    assert 2_000_000 <= waited < 1_000_000_000
    with pytest.raises(m.MbisError):
        m.mbis_debug_wait_timeout(0)
    w = workloads.tiny(n_samples=256)
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED)
    try:
        set_metric(m, ctx, prop)
        theta, _ = oracle.draw(spec.draw_seed, 0, 256, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        got = gpu_loglike(m, torch, ctx, theta)
        ref = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], theta, th))
        compare_loglike(got, ref, oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], theta))
    finally:
        m.mbis_destroy(ctx)
