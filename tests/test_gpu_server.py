"""Served stream: requests run to a target ESS under continuous admission, through the C ABI.

Each request's result must be the same alone (mbis_run_to_ess on a context of its own, with
relative binning set up the same way for a request that asks for it) and in a mix with
other requests on the device (bitwise: the request's arithmetic does not depend on what
else runs); admission must respect the HBM-footprint cap; a served
request's ESS and log Z must match the oracle's on the same draws (FP64: 1e-9 relative;
mixed precision: 1e-3 relative, the stated bound).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event, make_proposal
from gpu_common import m, torch, to_fp32_data  # noqa: F401

pytestmark = pytest.mark.gpu


def host_inputs(mod, ev, w, spec, th):
    if w.complex_dtype == "c64":
        strain, psd = to_fp32_data(ev)
    else:
        strain, psd = ev.strain[..., 0] + 1j * ev.strain[..., 1], ev.psd.copy()
    return dict(strain=strain, psd=psd, detectors=mod.make_detectors(ev.vertex, ev.xarm, ev.yarm), f_lo=w.f_lo,
                df=w.df, fixed=th, gmst=spec.gmst, marg=w.marg, n_tshift=w.n_tshift, dt_shift=w.dt_shift,
                dmin=w.dmin, dmax=w.dmax)


class Req:
    """One request: host inputs, proposal, precision and ESS-loop options."""

    rb = None

    def __init__(self, mod, w, spec, ev, th, prop, precision, ess_target, batch, max_samples, seed, refine=0,
                 refine_scale=0.0, rb=None):
        self.inp = host_inputs(mod, ev, w, spec, th)
        self.prop, self.precision = prop, precision
        self.rb = rb  # (fiducial, n_sigma, eps_rad): the ESS loop on relative binning
        self.ess = dict(ess_target=ess_target, batch=batch, max_samples=max_samples, seed=seed, refine=refine,
                        refine_scale=refine_scale)

    def submit(self, mod, server, tag=0):
        p = self.prop
        rb = {} if self.rb is None else dict(rb_fiducial=self.rb[0], rb_n_sigma=self.rb[1], rb_eps_rad=self.rb[2])
        return mod.mbis_server_submit(server, param_ids=p["ids"], mean=p["mean"], chol_lower=p["chol"],
                                      scale=p["scale"], prior_lo=p["lo"], prior_hi=p["hi"], prior_flags=p["flags"],
                                      precision=self.precision, tag=tag, **self.inp, **self.ess, **rb)

    def alone(self, mod, torch):
        i = self.inp
        ctx = mod.mbis_create(i["strain"], i["psd"], i["detectors"], i["f_lo"], i["df"], i["fixed"], gmst=i["gmst"],
                              precision=self.precision, marg=i["marg"], n_tshift=i["n_tshift"],
                              dt_shift=i["dt_shift"], dmin=i["dmin"], dmax=i["dmax"])
        try:
            p = self.prop
            mod.mbis_set_metric(ctx, p["ids"], p["mean"], p["chol"], p["scale"], p["lo"], p["hi"], p["flags"])
            if self.rb is not None:
                fid, ns, eps = self.rb
                edges = mod.mbis_rb_edges(ctx, fid, ns, eps, max_bins=len(i["psd"][0]))
                mod.mbis_rb_setup(ctx, fid, edges)
                mod.mbis_rb_use(ctx, True)
            P, b = len(p["ids"]), self.ess["batch"]
            bufs = [torch.empty((P, b), dtype=torch.float64, device="cuda")] + \
                   [torch.empty(b, dtype=torch.float64, device="cuda") for _ in range(4)]
            return mod.mbis_run_to_ess(ctx, *bufs, **self.ess)
        finally:
            mod.mbis_destroy(ctx)


@pytest.fixture(scope="module")
def requests(m):
    out = []
    w = workloads.tiny()
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    prop = make_proposal(ev, w, th)
    out.append(Req(m, w, spec, ev, th, prop, m.FP64, 2000.0, 1 << 14, 1 << 19, 11))
    out.append(Req(m, w, spec, ev, th, prop, m.MIXED, 2000.0, 1 << 14, 1 << 19, 12, refine=1, refine_scale=1.2))
    wb = workloads.scaled(workloads.bns_population(n_events=2), f_hi=512.0)
    rb_reqs = []
    for k, sp in enumerate(wb.events):
        evb, thb, _ = make_event(wb, sp)
        to_fp32_data(evb)
        propb = make_proposal(evb, wb, thb)
        out.append(Req(m, wb, sp, evb, thb, propb, m.MIXED, 1000.0, 1 << 15, 1 << 18, sp.draw_seed, refine=k))
        if k == 0:  # the same event with its ESS loop on relative binning about the injection
            rb_reqs.append(Req(m, wb, sp, evb, thb, propb, m.MIXED, 1000.0, 1 << 15, 1 << 18, sp.draw_seed,
                               refine=1, rb=(thb, 5.0, 0.1)))
    wt = workloads.bbh_population(n_events=1)
    sp = wt.events[0]
    evt, tht, _ = make_event(wt, sp)
    to_fp32_data(evt)
    out.append(Req(m, wt, sp, evt, tht, make_proposal(evt, wt, tht), m.MIXED, 1000.0, 1 << 14, 1 << 16,
                   sp.draw_seed, refine=1))
    return out + rb_reqs


def same(a, b):
    s, nd, nu = b
    assert a["status"] == 0, a["message"]
    assert a["n_drawn"] == nd and a["n_used"] == nu
    for k in ("ess", "log_z", "max_logw", "s1", "s2", "n"):
        assert a["summary"][k] == s[k] or (np.isnan(a["summary"][k]) and np.isnan(s[k])), k


def test_results_are_the_same_alone_and_in_the_mix(m, torch, requests):
    alone = [r.alone(m, torch) for r in requests]
    srv = m.mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=4)
    try:
        ids = [r.submit(m, srv, tag=k)[0] for k, r in enumerate(requests)]
        # a second copy of every request, submitted while the first ones run
        ids2 = [r.submit(m, srv, tag=100 + k)[0] for k, r in enumerate(requests)]
        res = [m.mbis_server_wait(srv, i, 300.0) for i in ids + ids2]
        st = m.mbis_server_stats_get(srv)
    finally:
        m.mbis_server_destroy(srv)
    n = len(requests)
    for k in range(n):
        assert res[k]["tag"] == k and res[n + k]["tag"] == 100 + k
        same(res[k], alone[k])
        same(res[n + k], alone[k])
        assert res[k]["t_submit"] <= res[k]["t_admit"] <= res[k]["t_done"]
    assert st["completed"] == 2 * n and st["failed"] == 0
    assert st["max_active_seen"] >= 2          # requests overlapped on the device
    assert st["max_active_seen"] <= 4 and st["active"] == 0 and st["bytes_in_use"] == 0


def test_admission_respects_the_hbm_cap(m, torch, requests):
    r = requests[2]
    probe = m.mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=1)
    try:
        _, fp = r.submit(m, probe)
    finally:
        m.mbis_server_destroy(probe)
    cap = int(2.5 * fp)                       # room for two requests of this shape
    srv = m.mbis_server_create(hbm_cap_bytes=cap, max_active=8)
    try:
        ids = [r.submit(m, srv, tag=k)[0] for k in range(6)]
        res = [m.mbis_server_wait(srv, i, 300.0) for i in ids]
        st = m.mbis_server_stats_get(srv)
    finally:
        m.mbis_server_destroy(srv)
    small = m.mbis_server_create(hbm_cap_bytes=fp // 100, max_active=1)
    try:
        with pytest.raises(m.MbisError):      # a request that can never fit is refused at once
            r.submit(m, small)
    finally:
        m.mbis_server_destroy(small)
    assert all(x["status"] == 0 for x in res)
    assert st["bytes_peak"] <= cap and st["max_active_seen"] == 2
    admits = [x["t_admit"] for x in res]
    assert admits == sorted(admits)           # first in, first out
    ref = res[0]["summary"]
    for x in res[1:]:
        assert x["summary"]["log_z"] == ref["log_z"]   # identical requests, identical results


def test_failed_request_reports_its_error_and_the_server_continues(m, torch, requests):
    srv = m.mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=2)
    try:
        bad = requests[0]
        inp = dict(bad.inp)
        inp["psd"] = inp["psd"].copy()
        inp["psd"][0, 3] = -1.0                # rejected when the context is made on the device side
        p = bad.prop
        rid, _ = m.mbis_server_submit(srv, param_ids=p["ids"], mean=p["mean"], chol_lower=p["chol"], scale=p["scale"],
                                      prior_lo=p["lo"], prior_hi=p["hi"], precision=m.FP64, **inp, **bad.ess)
        good, _ = requests[0].submit(m, srv)
        r_bad = m.mbis_server_wait(srv, rid, 300.0)
        r_good = m.mbis_server_wait(srv, good, 300.0)
        with pytest.raises(m.MbisError):
            m.mbis_server_wait(srv, rid, 1.0)  # already taken
    finally:
        m.mbis_server_destroy(srv)
    assert r_bad["status"] == m.MBIS_E_INVALID and "PSD" in r_bad["message"]
    same(r_good, requests[0].alone(m, torch))


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_served_request_matches_the_oracle(m, torch, requests, precision, rtol):
    """Two batches of 4096 with a fixed proposal: the served ESS and log Z against the
    oracle's draws, likelihoods and reduction of the same 8192 samples."""
    base = requests[0]
    r = Req.__new__(Req)
    r.inp, r.prop = base.inp, base.prop
    r.precision = m.FP64 if precision == "fp64" else m.MIXED
    r.ess = dict(ess_target=1e12, batch=4096, max_samples=8192, seed=77, refine=0, refine_scale=0.0)
    srv = m.mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=2)
    try:
        res = m.mbis_server_wait(srv, r.submit(m, srv)[0], 300.0)
    finally:
        m.mbis_server_destroy(srv)
    assert res["status"] == 0 and res["n_used"] == 8192 and res["n_drawn"] == 8192
    w = workloads.tiny()
    ev, th, _ = make_event(w, w.events[0])
    p = base.prop
    theta, lq = oracle.draw(77, 0, 8192, p["ids"], p["mean"], p["chol"], p["scale"])
    lp = oracle.log_prior(p["ids"], p["lo"], p["hi"], p["flags"], theta)
    ll = oracle.loglike_batch(ev, oracle.full_params(p["ids"], theta, th))
    want = oracle.reduce(ll, lp, lq)
    assert res["summary"]["ess"] == pytest.approx(want["ess"], rel=rtol)
    assert abs(res["summary"]["log_z"] - want["log_z"]) <= rtol


def test_relative_binning_requests_are_checked(m, torch, requests):
    """A served request's relative-binning parameters are checked at submission; asking for
    relative binning on a time-marginalised event (which it does not support) fails that
    request alone with MBIS_E_UNSUPPORTED, and the server goes on."""
    bns = requests[2]
    bbh = next(r for r in requests if r.inp["marg"] & m.MARG_TIME)
    srv = m.mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=2)
    try:
        for bad in (dict(rb_eps_rad=0.0), dict(rb_n_sigma=-1.0), dict(rb_max_bins=len(bns.inp["psd"][0]) + 1)):
            p = bns.prop
            kw = dict(rb_fiducial=bns.inp["fixed"], **bad)
            with pytest.raises(m.MbisError) as e:
                m.mbis_server_submit(srv, param_ids=p["ids"], mean=p["mean"], chol_lower=p["chol"], scale=p["scale"],
                                     prior_lo=p["lo"], prior_hi=p["hi"], prior_flags=p["flags"], precision=m.MIXED,
                                     **bns.inp, **bns.ess, **kw)
            assert e.value.status == m.MBIS_E_INVALID
        p = bbh.prop
        rid, _ = m.mbis_server_submit(srv, param_ids=p["ids"], mean=p["mean"], chol_lower=p["chol"], scale=p["scale"],
                                      prior_lo=p["lo"], prior_hi=p["hi"], prior_flags=p["flags"], precision=m.MIXED,
                                      rb_fiducial=bbh.inp["fixed"], **bbh.inp, **bbh.ess)
        good, _ = bns.submit(m, srv)
        r_bad = m.mbis_server_wait(srv, rid, 300.0)
        r_good = m.mbis_server_wait(srv, good, 300.0)
    finally:
        m.mbis_server_destroy(srv)
    assert r_bad["status"] == m.MBIS_E_UNSUPPORTED and "relative binning" in r_bad["message"]
    same(r_good, bns.alone(m, torch))
