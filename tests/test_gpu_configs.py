"""Evidence and effective sample size against the FP64 oracle per configuration, and the
kernel variants no other test input reaches.

Each case draws a batch on the device, evaluates it with the configuration's likelihood
kernel and reduces it (Eqs. 5-6); the oracle re-derives the same draws from its own
Philox, evaluates its own log L on them and reduces them itself.  Bounds: |delta log L|
<= 1e-3 per sample, relative ESS error <= 1e-3 and |delta log Z| <= 1e-3 (the stated
tolerances of the method); draws to 1e-12.

Variants covered here:
  * the BNS population (phase + distance marginalised, 128,513 bins), two events;
  * the 11-parameter BBH population (time marginalised on the tensor cores) at four mass
    pairs from 10 to 80 Msun, so that the live band runs from ~60 to ~1,600 bins and cuts
    fall on the 16-bin K-block boundaries;
  * the time-marginalised kernel with one folded detector row (fixed sky), two rows
    (H1+L1) and four rows (H1+L1+V1 and a fourth synthetic site);
  * FP64 entry of the anchor blocks (a coalescence time far from the reference time puts
    the t_c phase term above 2^16 turns) in the folded and the time-marginalised kernels.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import MC, Q, CHI1, CHI2, TC, PHIC
from oracle.events import make_event, make_proposal
from gpu_common import m, torch, gpu_context, set_metric, compare_loglike  # noqa: F401

pytestmark = pytest.mark.gpu

REL_ESS = 1e-3
ABS_LOGZ = 1e-3


def _with(spec, **kw):
    """A copy of an event spec with masses or slot values replaced."""
    import copy
    s = copy.deepcopy(spec)
    for k, v in kw.items():
        if k in ("m1", "m2", "snr"):
            setattr(s, k, v)
        else:
            s.params[k] = v
    return s


def run_case(m, torch, w, spec, n, precision=None, expect=None):
    """Draw n samples on the device, their log L and reduction, and the oracle's; compare.
    Returns (device log L, oracle log L, device summary, oracle summary, theta, info)."""
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    ctx = gpu_context(m, ev, w, spec, th, m.MIXED if precision is None else precision)
    try:
        set_metric(m, ctx, prop)
        info = m.mbis_get_info(ctx)
        for k, v in (expect or {}).items():
            assert info[k] == v, (k, info)
        P = len(prop["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq, lp, ll = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
        m.mbis_draw(ctx, spec.draw_seed, 0, n, theta, lq, lp)
        m.mbis_loglike(ctx, n, theta, ll)
        got = m.mbis_reduce(ctx, n, ll, lp, lq)
        torch.cuda.synchronize()
        th_d = theta.cpu().numpy()
        ref_th, ref_lq = oracle.draw(spec.draw_seed, 0, n, prop["ids"], prop["mean"], prop["chol"], prop["scale"])
        np.testing.assert_allclose(th_d, ref_th, rtol=1e-12, atol=1e-13)
        ref_lp = oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], ref_th)
        # a sample outside the prior has zero weight whatever its log L: the oracle
        # evaluates the samples inside
        inside = np.isfinite(ref_lp)
        ref_ll = np.zeros(n)
        ref_ll[inside] = oracle.loglike_batch(ev, oracle.full_params(prop["ids"], ref_th[:, inside], th))
        ll_d = ll.cpu().numpy()
        compare_loglike(ll_d, ref_ll, ref_lp)
        ref = oracle.reduce(ref_ll, ref_lp, ref_lq)
        assert got["n"] == ref["n"] == n
        print(f"  ESS {got['ess']:.4f} (oracle {ref['ess']:.4f}), log Z {got['log_z']:.6f} "
              f"(oracle {ref['log_z']:.6f}), {int(np.isfinite(ref_lp).sum())} of {n} in the prior, {info}")
        assert abs(got["ess"] / ref["ess"] - 1) <= REL_ESS, (got["ess"], ref["ess"])
        assert abs(got["log_z"] - ref["log_z"]) <= ABS_LOGZ, (got["log_z"], ref["log_z"])
        return ll_d, ref_ll, got, ref, ref_th, prop
    finally:
        m.mbis_destroy(ctx)


# ----------------------------------------------------------------------------- BNS population
@pytest.mark.parametrize("e", [0, 1])
def test_bns_evidence_matches_oracle(m, torch, e):
    w = workloads.bns_population(n_events=2, n_samples=1536)
    _, _, got, ref, th_s, prop = run_case(m, torch, w, w.events[e], 1536, expect=dict(tables=1, n_rows=1, ff_phase=1))
    assert int(np.isfinite(oracle.log_prior(prop["ids"], prop["lo"], prop["hi"], prop["flags"], th_s)).sum()) >= 512


# ----------------------------------------------------------------------------- BBH population
BBH_MASSES = [(12.0, 10.0), (31.0, 22.0), (55.0, 40.0), (70.0, 55.0)]


def _k_cut(w, mc, q):
    f = oracle.f_isco(mc, q)
    return max(0, min(w.n_bins, math.ceil((f - w.f_lo) / w.df)))


def test_bbh_evidence_matches_oracle_across_the_mass_range(m, torch):
    """Four events from light to heavy: the live band of the tensor-core contraction spans
    ~60 to ~1,600 bins; samples whose cut falls on a 16-bin K-block boundary are present."""
    w = workloads.bbh_population(n_events=4, n_samples=512)
    cuts = []
    for spec, (m1, m2) in zip(w.events, BBH_MASSES):
        s = _with(spec, m1=m1, m2=m2)
        _, _, _, _, th_s, prop = run_case(m, torch, w, s, 512, expect=dict(tables=0, n_rows=3, ff_phase=1))
        ids = list(prop["ids"])
        cuts += [_k_cut(w, th_s[ids.index(MC), i], th_s[ids.index(Q), i]) for i in range(th_s.shape[1])
                 if th_s[ids.index(Q), i] > 0 and th_s[ids.index(MC), i] > 0]
    cuts = np.array(cuts)
    on_boundary = int(np.sum((cuts > 0) & (cuts % 16 == 0)))
    print(f"  live bins per sample: {cuts.min()} .. {cuts.max()}, {on_boundary} end on a K-block boundary")
    assert cuts.min() < 100 and cuts.max() > 1400
    assert on_boundary >= 5


# ---------------------------------------------------------------- time kernel detector rows
def _synthetic_site():
    """A fourth detector for the four-row kernel: a site at 36.4 N, 137.3 E with arms along
    the local east and north (input data only; no real instrument is implied)."""
    lat, lon, r = math.radians(36.4), math.radians(137.3), 6.371e6
    up = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.cross(up, east)
    return dict(vertex=list(r * up), xarm=list(east), yarm=list(north))


@pytest.mark.parametrize("rows", [1, 2, 4])
def test_time_kernel_detector_rows(m, torch, monkeypatch, rows):
    """The time-marginalised kernel at the detector-row counts the BBH population does not
    use: fixed sky and orientation (one folded row), two detectors, four detectors."""
    monkeypatch.setitem(workloads.DETECTORS, "T1", _synthetic_site())
    w = workloads.bbh_population(n_events=2, n_samples=384)
    spec = _with(w.events[1], m1=24.0, m2=18.0)
    if rows == 1:
        w.sampled = [MC, Q, CHI1, CHI2, TC, PHIC]
    elif rows == 2:
        w.detectors = ["H1", "L1"]
    else:
        w.detectors = ["H1", "L1", "V1", "T1"]
    run_case(m, torch, w, spec, 384, expect=dict(n_rows=rows, ff_phase=1))


# ------------------------------------------------------------------- FP64 anchor-block entry
def test_fp64_block_entry_in_the_folded_kernel(m, torch):
    """A BNS event whose coalescence lies 300 s after the reference time: f t_c exceeds 2^16
    turns on a 20-256 Hz grid, so the folded kernel enters its anchor blocks in FP64."""
    w = workloads.scaled(workloads.bns_population(n_events=1, n_samples=512), f_hi=256.0)
    spec = _with(w.events[0], tc=300.0)
    run_case(m, torch, w, spec, 512, expect=dict(tables=1, ff_phase=0))


def test_fp64_block_entry_in_the_time_kernel(m, torch):
    """The same for the time-marginalised kernel: a BBH event at t_c = 100 s (f t_c up to
    1.02e5 turns on the 1024 Hz grid)."""
    w = workloads.bbh_population(n_events=1, n_samples=384)
    spec = _with(w.events[0], m1=30.0, m2=20.0, tc=100.0)
    run_case(m, torch, w, spec, 384, expect=dict(n_rows=3, ff_phase=0))
