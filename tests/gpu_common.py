"""Helpers shared by the GPU test modules: contexts built from oracle events, the FP32
rounding of the stored data, and the per-sample log L comparison."""
import os

import numpy as np
import pytest

LOGL_TOL = 1e-3


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
    # the observed error per case, for the per-configuration statement (pytest -s shows it)
    case = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    print(f"\n[log L vs oracle] {case}: max |delta| = {d.max():.2e}, "
          f"mean signed = {np.mean(got[inside] - ref[inside]):+.2e}, n = {int(inside.sum())}")
    assert d.max() <= LOGL_TOL, (d.max(), int(np.argmax(d)))
    return d.max()
