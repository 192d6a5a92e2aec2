"""mbis_reduce_noalloc: the weight reduction for callers that cannot allocate device memory
(a latency-critical loop, or a framework that owns all device memory).  Through the C ABI
it must give the same summary and weights as mbis_reduce (which keeps its scratch in a
context) and as the FP64 oracle, on calls in a row of falling size, treat NaN and -inf
log-weights as mbis_reduce does, and reject batches larger than its fixed scratch.

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


def _same(a, b):
    """Equal, counting NaN equal to NaN."""
    return (a == b) or (isinstance(a, float) and isinstance(b, float) and math.isnan(a) and math.isnan(b))


def test_noalloc_reduce_matches_the_oracle(m, torch):
    """Against the FP64 CPU reduction on the same inputs; a large call first, then a
    smaller one whose grid leaves most of the first call's partials in the array."""
    import oracle
    for seed, n in [(5, 1 << 22), (6, 3001), (7, 1)]:
        ll, lp, lq = _inputs(torch, seed, n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        got = m.mbis_reduce_noalloc(n, ll, lp, lq, w)
        ref = oracle.reduce(ll.cpu().numpy(), lp.cpu().numpy(), lq.cpu().numpy(), want_weights=True)
        assert got["n"] == ref["n"] == n and got["max_logw"] == ref["max_logw"]
        assert abs(got["ess"] / ref["ess"] - 1) < TOL
        assert abs(got["log_z"] - ref["log_z"]) < TOL * max(1.0, abs(ref["log_z"]))
        np.testing.assert_allclose(w.cpu().numpy(), ref["weights"], rtol=TOL, atol=1e-300)


def test_noalloc_reduce_treats_nan_and_inf_like_the_context_reduce(m, torch):
    """A NaN log-weight and -inf weights placed at and around the maximum: whatever the
    context reduction makes of them, the allocation-free one makes the same."""
    ctx = _context(m)
    try:
        n = 70_000
        ll, lp, lq = _inputs(torch, 11, n)
        k = int(torch.argmax(ll + lp - lq))
        lp[k + 1] = -math.inf               # next to the maximum
        lp[min(n - 1, k + 2048)] = -math.inf
        for poison in (None, float("nan")):
            if poison is not None:
                ll[n // 3] = poison
            w_ref = torch.empty(n, dtype=torch.float64, device="cuda")
            w_new = torch.empty(n, dtype=torch.float64, device="cuda")
            ref = m.mbis_reduce(ctx, n, ll, lp, lq, w_ref)
            got = m.mbis_reduce_noalloc(n, ll, lp, lq, w_new)
            for key in ("n", "max_logw", "all_zero"):
                assert _same(got[key], ref[key]), (poison, key, got[key], ref[key])
            for key in ("ess", "log_z", "s1", "s2"):
                a, b = got[key], ref[key]
                assert _same(a, b) or abs(a - b) <= TOL * max(1.0, abs(b)), (poison, key, a, b)
            a, b = w_new.cpu().numpy(), w_ref.cpu().numpy()
            assert np.array_equal(np.isnan(a), np.isnan(b))
            np.testing.assert_allclose(a[~np.isnan(a)], b[~np.isnan(b)], rtol=TOL, atol=1e-300)
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
