"""The device Fisher matrix (mbis_fisher) and the proposal built behind the C ABI
(mbis_fisher_proposal) against the oracle's Fisher matrix and the test side's recipe."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, make_proposal, marginalised_slots, fisher_steps
from gpu_common import m, torch, gpu_context  # noqa: F401

pytestmark = pytest.mark.gpu


def _cases():
    tiny = workloads.tiny(n_samples=16)
    bns = workloads.scaled(workloads.bns_population(n_events=2, n_samples=16), f_hi=256.0)
    bbh = workloads.bbh_population(n_events=3, n_samples=16)
    return [("tiny", tiny, tiny.events[0]), ("bns", bns, bns.events[0]), ("bbh", bbh, bbh.events[2])]


@pytest.mark.parametrize("name,w,spec", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_fisher_and_proposal_match_the_oracle(m, torch, name, w, spec):
    ev, th, _ = make_event(w, spec)
    ctx = gpu_context(m, ev, w, spec, th, m.FP64)
    try:
        ids = list(w.sampled) + marginalised_slots(w.marg)
        steps = fisher_steps(ids, th)
        got = m.mbis_fisher(ctx, th, ids, steps)
        ref = oracle.fisher(ev.with_marg(0), th, ids, steps)
        # both sides difference FP64 waveforms with the same steps: agreement to ~1e-8 of the
        # matrix scale (central differences lose half the digits of each waveform value)
        scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.max(np.abs(got - ref) / scale) < 1e-6, np.max(np.abs(got - ref) / scale)
        prop = m.fisher_proposal(ctx, th, w.sampled, scale=w.scale, box_sigmas=w.box_sigmas, chi_max=w.chi_max,
                                 dmin=w.dmin, dmax=w.dmax, prior_flags=w.prior_flags)
        rp = make_proposal(ev, w, th)
        np.testing.assert_array_equal(prop["mean"], rp["mean"])
        cg, cr = prop["chol"] @ prop["chol"].T, rp["chol"] @ rp["chol"].T
        sd = np.sqrt(np.outer(np.diag(cr), np.diag(cr)))
        assert np.max(np.abs(cg - cr) / sd) < 1e-4, np.max(np.abs(cg - cr) / sd)
        np.testing.assert_allclose(prop["lo"], rp["lo"], rtol=1e-5, atol=1e-12)
        np.testing.assert_allclose(prop["hi"], rp["hi"], rtol=1e-5, atol=1e-12)
        # the proposal is accepted by mbis_set_metric as it comes
        m.mbis_set_metric(ctx, prop["ids"], prop["mean"], prop["chol"], prop["scale"], prop["lo"], prop["hi"],
                          prop["flags"])
    finally:
        m.mbis_destroy(ctx)
