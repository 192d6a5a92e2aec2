"""mbis_reduce_noalloc: the weight reduction for callers that cannot allocate device memory
(a latency-critical loop, or a framework that owns all device memory).  Through the C ABI
it must give the same summary and weights as mbis_reduce (which keeps its scratch in a
context), on two calls in a row, and reject batches larger than its fixed scratch.

This file sorts last so that a run stopping at the first failure has already run every
other test; it also passes when run alone in a fresh process."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the tolerance of the reduction-only comparisons in the parity tests


@pytest.fixture(scope="module")
def m():
    import paper_2410_05190_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _inputs(torch, seed, n):
    rng = np.random.default_rng(seed)
    ll = rng.normal(40.0, 6.0, n)
    lp = np.where(rng.uniform(size=n) < 0.05, -np.inf, rng.normal(-2.0, 0.5, n))
    lq = rng.normal(-1.0, 1.0, n)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    return T(ll), T(lp), T(lq)


def _context(m):
    """A minimal context: mbis_reduce needs one for its scratch."""
    n_bins = 8
    dets = m.make_detectors([[0.0, 0.0, 6.4e6]], [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    strain = np.zeros((1, n_bins), dtype=np.complex128)
    psd = np.ones((1, n_bins))
    fixed = [1.2, 1.1, 0, 0, 0, 0, 0, 0, 100.0, 0, 0]
    return m.mbis_create(strain, psd, dets, 20.0, 1.0, fixed, precision=m.FP64, marg=m.MARG_PHASE)


def test_noalloc_reduce_matches_the_context_reduce_on_two_calls(m, torch):
    ctx = _context(m)
    try:
        for seed, n in [(1, 300_001), (2, 4097)]:   # second call: different size and contents
            ll, lp, lq = _inputs(torch, seed, n)
            w_ref = torch.empty(n, dtype=torch.float64, device="cuda")
            w_new = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            ref = m.mbis_reduce(ctx, n, ll, lp, lq, w_ref)
            got = m.mbis_reduce_noalloc(n, ll, lp, lq, w_new)
            assert got["n"] == ref["n"] == n
            assert got["max_logw"] == ref["max_logw"]
            assert abs(got["ess"] / ref["ess"] - 1) < TOL
            assert abs(got["log_z"] - ref["log_z"]) < TOL * max(1.0, abs(ref["log_z"]))
            np.testing.assert_allclose(w_new.cpu().numpy(), w_ref.cpu().numpy(), rtol=TOL, atol=1e-300)
    finally:
        m.mbis_destroy(ctx)


def test_noalloc_reduce_edge_cases(m, torch):
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    s = m.mbis_reduce_noalloc(0, z, z, z)
    assert s["n"] == 0 and s["ess"] == 0 and s["all_zero"]
    n = 5000
    ninf = torch.full((n,), -math.inf, dtype=torch.float64, device="cuda")
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = m.mbis_reduce_noalloc(n, ninf, zero, zero)
    assert s["ess"] == 0 and s["log_z"] == -math.inf and s["all_zero"]
    with pytest.raises(m.MbisError) as e:
        m.mbis_reduce_noalloc(m.NOALLOC_MAX_SAMPLES + 1, zero, zero, zero)
    assert e.value.status == m.MBIS_E_INVALID
    assert str(m.NOALLOC_MAX_SAMPLES) in str(e.value)
