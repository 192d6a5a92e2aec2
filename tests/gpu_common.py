"""Helpers shared by the GPU test modules: contexts built from oracle events, the FP32
rounding of the stored data, and the per-sample log L comparison."""
import os

import numpy as np
import pytest

LOGL_TOL = 1e-3
# Below log L = -LOGL_SCALE the bound grows in proportion to |log L|: such a sample's weight
# is under e^(-1000) of that of any sample near the likelihood peak (log L >= 0; every event
# here peaks above 50) -- zero in double precision, whatever its log L -- while the FP32
# contractions' error is relative to the overlap |z| (FP32 holds |z| = 6e4 to 4e-3).
LOGL_SCALE = 1e3


def logl_bound(ref):
    """Per-sample bound on |delta log L|: 1e-3, or 1e-3 per 10^3 of |log L| below -10^3."""
    return LOGL_TOL * np.maximum(1.0, -np.asarray(ref) / LOGL_SCALE)


@pytest.fixture(scope="module")
def m():
    import paper_2410_05190_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def to_fp32_data(ev):
    """Round an oracle event's data to the complex64 the GPU stores (the PSD stays FP64)."""
    s = (ev.strain[..., 0] + 1j * ev.strain[..., 1]).astype(np.complex64)
    ev.set_strain(np.stack([s.real.astype(np.float64), s.imag.astype(np.float64)], axis=-1))
    return s, ev.psd.copy()


def gpu_context(m, ev, w, spec, th, precision):
    if w.complex_dtype == "c64":
        strain, psd = to_fp32_data(ev)
    else:
        strain, psd = ev.strain[..., 0] + 1j * ev.strain[..., 1], ev.psd.copy()
    dets = m.make_detectors(ev.vertex, ev.xarm, ev.yarm)
    return m.mbis_create(strain, psd, dets, w.f_lo, w.df, th, gmst=spec.gmst, precision=precision, marg=w.marg,
                         n_tshift=w.n_tshift, dt_shift=w.dt_shift, dmin=w.dmin, dmax=w.dmax)


def set_metric(m, ctx, prop):
    m.mbis_set_metric(ctx, prop["ids"], prop["mean"], prop["chol"], prop["scale"], prop["lo"], prop["hi"],
                      prop["flags"])


def gpu_loglike(m, torch, ctx, theta_soa):
    th = torch.tensor(np.ascontiguousarray(theta_soa), dtype=torch.float64, device="cuda")
    n = th.shape[1]
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    m.mbis_loglike(ctx, n, th, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def compare_loglike(got, ref, logp):
    inside = np.isfinite(logp)
    assert np.all(np.isfinite(ref[inside]))
    d = np.abs(got[inside] - ref[inside])
    bound = logl_bound(ref[inside])
    near = ref[inside] >= -LOGL_SCALE
    # the observed error per case, for the per-configuration statement (pytest -s shows it)
    case = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    far = "" if near.all() else (f"; log L < -1e3: {int((~near).sum())} samples, max |delta| = {d[~near].max():.2e}, "
                                 f"max |delta / log L| = {np.max(d[~near] / np.abs(ref[inside][~near])):.1e}")
    print(f"\n[log L vs oracle] {case}: max |delta| = {d[near].max() if near.any() else 0.0:.2e}, "
          f"mean signed = {np.mean((got[inside] - ref[inside])[near]) if near.any() else 0.0:+.2e}, "
          f"n = {int(near.sum())}{far}")
    assert np.all(d <= bound), (d.max(), int(np.argmax(d / bound)), ref[inside][int(np.argmax(d / bound))])
    return d[near].max() if near.any() else 0.0
