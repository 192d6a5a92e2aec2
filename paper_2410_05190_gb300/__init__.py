"""GB300-native metric-based importance sampling for compact-binary parameter estimation.

Thin Python binding over the C ABI of ``libmbis.so`` (declared in ``include/mbis.h``):
the functions below carry the same names as the C entry points and only marshal
arguments (numpy arrays for host buffers, torch tensors or raw integers for device
buffers and streams).  Every step of the computation runs in the library's CUDA kernels.
Importing this package fails loudly when the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB

MBIS_OK, MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA, MBIS_E_TIMEOUT, MBIS_E_STATE, MBIS_E_UNSUPPORTED = range(7)
STATUS_NAMES = ["MBIS_OK", "MBIS_E_INVALID", "MBIS_E_OOM", "MBIS_E_CUDA", "MBIS_E_TIMEOUT", "MBIS_E_STATE",
                "MBIS_E_UNSUPPORTED"]
P_MC, P_Q, P_CHI1, P_CHI2, P_RA, P_DEC, P_PSI, P_IOTA, P_DL, P_TC, P_PHIC = range(11)
NPAR = 11
MARG_PHASE, MARG_DISTANCE, MARG_TIME = 1, 2, 4
C128, C64 = 0, 1
FP64, MIXED = 0, 1
PRIOR_M1M2 = 1


class MbisError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status


class FreqGrid(C.Structure):
    _fields_ = [("f_lo", C.c_double), ("df", C.c_double), ("n_bins", C.c_int32)]


class Detector(C.Structure):
    _fields_ = [("vertex_m", C.c_double * 3), ("xarm", C.c_double * 3), ("yarm", C.c_double * 3)]


class Event(C.Structure):
    _fields_ = [("n_det", C.c_int32), ("dtype", C.c_int32), ("strain", C.c_void_p), ("gmst_rad", C.c_double),
                ("fixed", C.c_double * 11)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("marg", C.c_uint32), ("n_tshift", C.c_int32), ("dt_shift", C.c_double),
                ("dmin_mpc", C.c_double), ("dmax_mpc", C.c_double)]


class ProposalOptions(C.Structure):
    _fields_ = [("scale", C.c_double), ("box_sigmas", C.c_double), ("chi_max", C.c_double),
                ("dmin_mpc", C.c_double), ("dmax_mpc", C.c_double)]


class CtxInfo(C.Structure):
    _fields_ = [("tables", C.c_int32), ("n_rows", C.c_int32), ("ff_phase", C.c_int32), ("n_blocks", C.c_int32),
                ("P", C.c_int32)]


class Summary(C.Structure):
    _fields_ = [("ess", C.c_double), ("log_z", C.c_double), ("max_logw", C.c_double), ("n", C.c_int64),
                ("s1", C.c_double), ("s2", C.c_double), ("all_zero", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EssOptions(C.Structure):
    _fields_ = [("ess_target", C.c_double), ("batch", C.c_int64), ("max_samples", C.c_int64), ("refine", C.c_int32),
                ("refine_scale", C.c_double), ("seed", C.c_uint64), ("refit_min_ess", C.c_double)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_cap_bytes", C.c_int64), ("max_active", C.c_int32), ("device", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("event", Event), ("psd", C.c_void_p), ("dets", C.c_void_p), ("grid", FreqGrid), ("opts", Options),
                ("P", C.c_int32), ("ids", C.c_void_p), ("mean", C.c_void_p), ("chol", C.c_void_p),
                ("scale", C.c_double), ("lo", C.c_void_p), ("hi", C.c_void_p), ("prior_flags", C.c_uint32),
                ("ess", EssOptions), ("tag", C.c_uint64), ("rb_fiducial", C.c_void_p), ("rb_n_sigma", C.c_double),
                ("rb_eps_rad", C.c_double), ("rb_max_bins", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int32), ("pad", C.c_int32),
                ("summary", Summary), ("n_drawn", C.c_int64), ("n_used", C.c_int64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("footprint_bytes", C.c_int64),
                ("message", C.c_char * 160)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "summary", "message")}
        d["summary"] = self.summary.as_dict()
        d["message"] = self.message.decode(errors="replace")
        return d


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("bytes_in_use", C.c_int64), ("bytes_peak", C.c_int64),
                ("bytes_cap", C.c_int64), ("max_active_seen", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    p, i32, i64, u32, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    sigs = {
        "mbis_create": [p, p, p, p, p, p],
        "mbis_set_metric": [p, i32, p, p, p, d, p, p, u32],
        "mbis_draw": [p, u64, u64, i64, p, p, p, p],
        "mbis_loglike": [p, i64, p, p, p],
        "mbis_reduce": [p, i64, p, p, p, p, i32, p, p],
        "mbis_get_running": [p, p],
        "mbis_reset_running": [p],
        "mbis_psd_aligo": [p, p],
        "mbis_inject": [p, i32, p, p, d, p, u64, i32, p, p],
        "mbis_fisher": [p, p, i32, p, p, p],
        "mbis_proposal_from_fisher": [i32, p, i32, p, p, p, p, p, p, p, p],
        "mbis_fisher_proposal": [p, p, i32, p, p, p, p, p, p],
        "mbis_reduce_noalloc": [i64, p, p, p, p, p, p],
        "mbis_weighted_moments": [p, i64, p, p, p, p, p],
        "mbis_set_proposal": [p, p, p, d],
        "mbis_get_proposal": [p, p, p, p],
        "mbis_get_info": [p, p],
        "mbis_run_to_ess": [p, p, p, p, p, p, p, p, p, p, p],
        "mbis_batch_create": [i32, p, p, p, p],
        "mbis_batch_step": [p, u64, p],
        "mbis_batch_autotune": [p, p, p],
        "mbis_batch_shape": [p, p, p],
        "mbis_batch_set_shape": [p, i32, i32],
        "mbis_batch_loglike": [p, p],
        "mbis_batch_buffers": [p, i32, p, p],
        "mbis_batch_copy_out": [p, i32, p, p],
        "mbis_server_create": [p, p],
        "mbis_server_submit": [p, p, p, p],
        "mbis_server_wait": [p, u64, d, p],
        "mbis_server_poll": [p, p, i32, p],
        "mbis_server_stats_get": [p, p],
        "mbis_debug_wait_timeout": [u64, p, p],
        "mbis_debug_ff_sincos": [i64, p, p, p, p],
        "mbis_debug_setup_pair": [i64, p, d, d, i32, p, p],
        "mbis_credible_levels": [i64, i32, p, p, p, p, p],
        "mbis_rb_setup": [p, p, i32, p],
        "mbis_rb_loglike": [p, i64, p, p, p],
        "mbis_rb_edges": [p, p, d, d, i32, p, p],
        "mbis_rb_use": [p, i32],
        "mbis_tiling_create": [p, p, p, p],
        "mbis_tiling_bank": [p, i64, p, d, i64, i32, p, p],
        "mbis_tiling_templates": [p, p, p, p, p],
        "mbis_tiling_match": [p, i64, p, p, p, p],
        "mbis_tiling_assign": [p, i64, p, p, p, p],
        "mbis_tiling_set_pool": [p, i64, p, p],
        "mbis_tiling_pool": [p, p, p, p, p],
        "mbis_tiling_set_loglike": [p, p, p],
        "mbis_tiling_draw": [p, u64, u64, i64, p, p, p, p, p, p],
    }
    lib.mbis_tiling_destroy.restype = None
    lib.mbis_tiling_destroy.argtypes = [p]
    lib.mbis_tiling_last_error.restype = C.c_char_p
    lib.mbis_tiling_last_error.argtypes = [p]
    lib.mbis_server_destroy.restype = None
    lib.mbis_server_destroy.argtypes = [p]
    lib.mbis_batch_destroy.restype = None
    lib.mbis_batch_destroy.argtypes = [p]
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.restype = C.c_int
        f.argtypes = args
    lib.mbis_merge_summaries.restype = None
    lib.mbis_merge_summaries.argtypes = [p, p, p]
    lib.mbis_destroy.restype = None
    lib.mbis_destroy.argtypes = [p]
    lib.mbis_last_error.restype = C.c_char_p
    lib.mbis_last_error.argtypes = [p]
    lib.mbis_version.restype = C.c_char_p
    lib.mbis_version.argtypes = []
    return lib


_lib = _load()


def lib():
    return _lib


def _check(status, ctx=None):
    if status != MBIS_OK:
        msg = _lib.mbis_last_error(ctx)
        raise MbisError(status, msg.decode() if msg else "")


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _dev(x):
    """Device pointer of a torch tensor (or a raw integer address); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_detectors(vertex, xarm, yarm):
    n = len(vertex)
    arr = (Detector * n)()
    for d in range(n):
        arr[d].vertex_m[:] = list(map(float, vertex[d]))
        arr[d].xarm[:] = list(map(float, xarm[d]))
        arr[d].yarm[:] = list(map(float, yarm[d]))
    return arr


# ------------------------------------------------------------------------------- entry points
def mbis_create(strain, psd, detectors, f_lo, df, fixed, gmst=0.0, precision=MIXED, marg=MARG_PHASE, n_tshift=128,
                dt_shift=1e-4, dmin=10.0, dmax=1000.0):
    """strain: complex host array [n_det, n_bins] (complex128 or complex64); psd: float64
    host array [n_det, n_bins]; detectors: ctypes array from make_detectors; fixed: 11
    slot values.  Returns the context handle (int)."""
    strain = np.ascontiguousarray(strain)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    if strain.dtype == np.complex128:
        dtype = C128
    elif strain.dtype == np.complex64:
        dtype = C64
    else:
        raise TypeError("strain must be complex128 or complex64")
    n_det, n_bins = strain.shape
    ev = Event(n_det, dtype, strain.ctypes.data, gmst, (C.c_double * 11)(*map(float, fixed)))
    grid = FreqGrid(f_lo, df, n_bins)
    opts = Options(precision, marg, n_tshift, dt_shift, dmin, dmax)
    out = C.c_void_p()
    _check(_lib.mbis_create(C.byref(ev), psd.ctypes.data, detectors, C.byref(grid), C.byref(opts), C.byref(out)))
    return out.value


def mbis_set_metric(ctx, param_ids, mean, chol_lower, scale, prior_lo, prior_hi, prior_flags=0):
    ids, pid = _host(param_ids, np.int32)
    m, pm = _host(mean, np.float64)
    L, pL = _host(chol_lower, np.float64)
    lo, plo = _host(prior_lo, np.float64)
    hi, phi = _host(prior_hi, np.float64)
    _check(_lib.mbis_set_metric(ctx, len(ids), pid, pm, pL, scale, plo, phi, prior_flags), ctx)


def mbis_draw(ctx, seed, ctr0, n, theta, log_q=None, log_prior=None, stream=None):
    _check(_lib.mbis_draw(ctx, seed, ctr0, n, _dev(theta), _dev(log_q), _dev(log_prior), _stream(stream)), ctx)


def mbis_loglike(ctx, n, theta, loglike, stream=None):
    _check(_lib.mbis_loglike(ctx, n, _dev(theta), _dev(loglike), _stream(stream)), ctx)


def mbis_reduce(ctx, n, loglike, log_prior, log_q, weights_out=None, accumulate=False, stream=None):
    out = Summary()
    _check(_lib.mbis_reduce(ctx, n, _dev(loglike), _dev(log_prior), _dev(log_q), _dev(weights_out), int(accumulate),
                            C.byref(out), _stream(stream)), ctx)
    return out.as_dict()


def mbis_weighted_moments(ctx, n, theta, weights, stream=None):
    """Returns (mean [P], covariance [P, P]) of the weighted samples."""
    P = len(theta) if not isinstance(theta, int) else None
    mean = np.zeros(11)
    cov = np.zeros(121)
    _check(_lib.mbis_weighted_moments(ctx, n, _dev(theta), _dev(weights), mean.ctypes.data, cov.ctypes.data,
                                      _stream(stream)), ctx)
    if P is None:
        raise ValueError("pass theta as a [P, n] tensor")
    return mean[:P].copy(), cov[:P * P].reshape(P, P).copy()


def mbis_set_proposal(ctx, mean, chol_lower, scale):
    m, pm = _host(mean, np.float64)
    L, pL = _host(chol_lower, np.float64)
    _check(_lib.mbis_set_proposal(ctx, pm, pL, scale), ctx)


def mbis_get_info(ctx):
    """What mbis_set_metric built: tables (1 folded, 0 per detector, -1 none), n_rows,
    ff_phase (1 float-float block entry, 0 FP64, -1 not mixed), n_blocks, P."""
    out = CtxInfo()
    _check(_lib.mbis_get_info(ctx, C.byref(out)))
    return {k: getattr(out, k) for k, _ in out._fields_}


def mbis_get_proposal(ctx, P):
    """The context's current proposal over its P sampled slots: (mean [P], chol [P, P], scale)."""
    mean, chol, sc = np.zeros(11), np.zeros(121), C.c_double()
    _check(_lib.mbis_get_proposal(ctx, mean.ctypes.data, chol.ctypes.data, C.byref(sc)), None if ctx is None else ctx)
    return mean[:P].copy(), chol[:P * P].reshape(P, P).copy(), sc.value


def mbis_run_to_ess(ctx, theta, log_q, log_prior, loglike, weights, ess_target, batch, max_samples, seed, refine=0,
                    refine_scale=0.0, stream=None, refit_min_ess=0.0):
    """Returns (summary dict, n_drawn, n_used)."""
    opts = EssOptions(ess_target, batch, max_samples, refine, refine_scale, seed, refit_min_ess)
    out = Summary()
    nd, nu = C.c_int64(), C.c_int64()
    _check(_lib.mbis_run_to_ess(ctx, C.byref(opts), _dev(theta), _dev(log_q), _dev(log_prior), _dev(loglike),
                                _dev(weights), C.byref(out), C.byref(nd), C.byref(nu), _stream(stream)), ctx)
    return out.as_dict(), nd.value, nu.value


def mbis_batch_create(ctxs, n_samples, seeds):
    n = len(ctxs)
    arr = (C.c_void_p * n)(*ctxs)
    ns = np.ascontiguousarray(n_samples, dtype=np.int64)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    out = C.c_void_p()
    _check(_lib.mbis_batch_create(n, arr, ns.ctypes.data, sd.ctypes.data, C.byref(out)))
    return out.value


def mbis_batch_step(b, step, n_ctx):
    out = (Summary * n_ctx)()
    _check(_lib.mbis_batch_step(b, step, out))
    return [s.as_dict() for s in out]


def mbis_batch_autotune(b):
    g, ms = C.c_int32(), C.c_float()
    _check(_lib.mbis_batch_autotune(b, C.byref(g), C.byref(ms)))
    return g.value, ms.value


def mbis_batch_set_shape(b, samples_per_cta, ctas_per_sm):
    _check(_lib.mbis_batch_set_shape(b, samples_per_cta, ctas_per_sm))


def mbis_batch_shape(b):
    """(samples per CTA, CTAs in the grid) of the batch's persistent launch."""
    t, g = C.c_int32(), C.c_int32()
    _check(_lib.mbis_batch_shape(b, C.byref(t), C.byref(g)))
    return t.value, g.value


def mbis_batch_loglike(b, stream=None):
    _check(_lib.mbis_batch_loglike(b, _stream(stream)))


def mbis_batch_buffers(b, i):
    th, ll = C.c_void_p(), C.c_void_p()
    _check(_lib.mbis_batch_buffers(b, i, C.byref(th), C.byref(ll)))
    return th.value, ll.value


def mbis_batch_copy_out(b, i, P, n):
    th = np.zeros((P, n))
    ll = np.zeros(n)
    _check(_lib.mbis_batch_copy_out(b, i, th.ctypes.data, ll.ctypes.data))
    return th, ll


def mbis_batch_destroy(b):
    _lib.mbis_batch_destroy(b)


def mbis_server_create(hbm_cap_bytes=150 * 10**9, max_active=8, device=0):
    out = C.c_void_p()
    opts = ServerOptions(int(hbm_cap_bytes), max_active, device)
    _check(_lib.mbis_server_create(C.byref(opts), C.byref(out)))
    return out.value


def mbis_server_submit(server, strain, psd, detectors, f_lo, df, fixed, param_ids, mean, chol_lower, scale,
                       prior_lo, prior_hi, prior_flags=0, gmst=0.0, precision=MIXED, marg=MARG_PHASE, n_tshift=128,
                       dt_shift=1e-4, dmin=10.0, dmax=1000.0, ess_target=1e4, batch=1 << 16, max_samples=1 << 24,
                       seed=0, refine=0, refine_scale=0.0, tag=0, rb_fiducial=None, rb_n_sigma=5.0, rb_eps_rad=0.3,
                       rb_max_bins=None, refit_min_ess=0.0):
    """Queue one request (the arguments of mbis_create, mbis_set_metric and
    mbis_run_to_ess; rb_fiducial (11 slots) runs its ESS loop on relative binning about it).
    Returns (request id, footprint bytes)."""
    strain = np.ascontiguousarray(strain)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    if strain.dtype == np.complex128:
        dtype = C128
    elif strain.dtype == np.complex64:
        dtype = C64
    else:
        raise TypeError("strain must be complex128 or complex64")
    n_det, n_bins = strain.shape
    ids, pid = _host(param_ids, np.int32)
    m, pm = _host(mean, np.float64)
    L, pL = _host(chol_lower, np.float64)
    lo, plo = _host(prior_lo, np.float64)
    hi, phi = _host(prior_hi, np.float64)
    req = Request(Event(n_det, dtype, strain.ctypes.data, gmst, (C.c_double * 11)(*map(float, fixed))),
                  psd.ctypes.data, C.cast(detectors, C.c_void_p), FreqGrid(f_lo, df, n_bins),
                  Options(precision, marg, n_tshift, dt_shift, dmin, dmax), len(ids), pid, pm, pL, scale, plo, phi,
                  prior_flags, EssOptions(ess_target, batch, max_samples, refine, refine_scale, seed, refit_min_ess), tag)
    if rb_fiducial is not None:
        fid, pfid = _host(rb_fiducial, np.float64)
        req.rb_fiducial, req.rb_n_sigma, req.rb_eps_rad = pfid, rb_n_sigma, rb_eps_rad
        req.rb_max_bins = n_bins if rb_max_bins is None else rb_max_bins
    rid, fp = C.c_uint64(), C.c_int64()
    _check(_lib.mbis_server_submit(server, C.byref(req), C.byref(rid), C.byref(fp)))
    return rid.value, fp.value


def mbis_server_wait(server, rid, timeout=-1.0):
    out = Result()
    _check(_lib.mbis_server_wait(server, rid, timeout, C.byref(out)))
    return out.as_dict()


def mbis_server_poll(server, max_results=64):
    out = (Result * max_results)()
    n = C.c_int32()
    _check(_lib.mbis_server_poll(server, out, max_results, C.byref(n)))
    return [out[i].as_dict() for i in range(n.value)]


def mbis_server_stats_get(server):
    out = ServerStats()
    _check(_lib.mbis_server_stats_get(server, C.byref(out)))
    return out.as_dict()


def mbis_server_destroy(server):
    _lib.mbis_server_destroy(server)


def mbis_debug_wait_timeout(limit_ns):
    """Returns (status, waited_ns) of a device wait on a barrier that never completes."""
    st, ns = C.c_int32(), C.c_uint64()
    _check(_lib.mbis_debug_wait_timeout(int(limit_ns), C.byref(st), C.byref(ns)))
    return st.value, ns.value


def mbis_debug_ff_sincos(n, x, sin_out=None, cos_out=None, stream=None):
    """The time kernel's float-float sine and cosine of n device angles (a self-test)."""
    _check(_lib.mbis_debug_ff_sincos(int(n), _dev(x), _dev(sin_out), _dev(cos_out), _stream(stream)))


def mbis_debug_setup_pair(n, params, f_lo, df, n_bins, out, stream=None):
    """FP64 and float-float per-sample set-up side by side (a self-test; out [2][12][n])."""
    _check(_lib.mbis_debug_setup_pair(int(n), _dev(params), float(f_lo), float(df), int(n_bins), _dev(out),
                                      _stream(stream)))


NOALLOC_MAX_SAMPLES = 16777216


def mbis_reduce_noalloc(n, loglike, log_prior, log_q, weights_out=None, stream=None):
    """The reduction without a context or any allocation (see include/mbis.h)."""
    out = Summary()
    _check(_lib.mbis_reduce_noalloc(n, _dev(loglike), _dev(log_prior), _dev(log_q), _dev(weights_out), C.byref(out),
                                    _stream(stream)))
    return out.as_dict()


def mbis_get_running(ctx):
    out = Summary()
    _check(_lib.mbis_get_running(ctx, C.byref(out)), ctx)
    return out.as_dict()


def mbis_reset_running(ctx):
    _check(_lib.mbis_reset_running(ctx), ctx)


def mbis_merge_summaries(a: dict, b: dict):
    sa = Summary(**a)
    sb = Summary(**b)
    out = Summary()
    _lib.mbis_merge_summaries(C.byref(sa), C.byref(sb), C.byref(out))
    return out.as_dict()


def mbis_destroy(ctx):
    _lib.mbis_destroy(ctx)


def mbis_last_error(ctx=None):
    m = _lib.mbis_last_error(ctx)
    return m.decode() if m else ""


def mbis_version():
    return _lib.mbis_version().decode()


def mbis_psd_aligo(f_lo, df, n_bins):
    out = np.zeros(n_bins)
    grid = FreqGrid(f_lo, df, n_bins)
    _check(_lib.mbis_psd_aligo(C.byref(grid), out.ctypes.data))
    return out


def mbis_inject(f_lo, df, n_bins, detectors, psd, gmst, theta_true, noise_seed=0, add_noise=False):
    """Returns (strain complex128 [n_det, n_bins], optimal SNR^2)."""
    n_det = len(detectors)
    psd = np.ascontiguousarray(psd, dtype=np.float64).reshape(n_det, n_bins)
    th, pth = _host(theta_true, np.float64)
    out = np.zeros((n_det, n_bins), dtype=np.complex128)
    snr2 = C.c_double()
    grid = FreqGrid(f_lo, df, n_bins)
    _check(_lib.mbis_inject(C.byref(grid), n_det, detectors, psd.ctypes.data, gmst, pth, noise_seed, int(add_noise),
                            out.ctypes.data, C.byref(snr2)))
    return out, snr2.value


def mbis_fisher(ctx, theta, ids, steps):
    th, pth = _host(theta, np.float64)
    ids, pid = _host(ids, np.int32)
    st, pst = _host(steps, np.float64)
    P = len(ids)
    g = np.zeros((P, P))
    _check(_lib.mbis_fisher(ctx, pth, P, pid, pst, g.ctypes.data), ctx)
    return g


def _proposal_dict(ids, mean, chol, lo, hi, scale, prior_flags):
    return dict(ids=ids, mean=mean, chol=chol, scale=scale, lo=lo, hi=hi, flags=prior_flags)


def mbis_proposal_from_fisher(ids, marg_ids, gamma, theta0, scale=1.5, box_sigmas=10.0, chi_max=0.99, dmin=10.0,
                              dmax=1000.0, prior_flags=0):
    """Proposal dict (ids, mean, chol, scale, lo, hi, flags) for mbis_set_metric from a
    Fisher matrix over ids + marg_ids (host arithmetic in the library; no GPU needed)."""
    ids, pid = _host(ids, np.int32)
    mids, pmid = _host(marg_ids, np.int32)
    g, pg = _host(gamma, np.float64)
    th, pth = _host(theta0, np.float64)
    P = len(ids)
    mean, chol, lo, hi = np.zeros(P), np.zeros((P, P)), np.zeros(P), np.zeros(P)
    o = ProposalOptions(scale, box_sigmas, chi_max, dmin, dmax)
    _check(_lib.mbis_proposal_from_fisher(P, pid, len(mids), pmid if len(mids) else None, pg, pth, C.byref(o),
                                          mean.ctypes.data, chol.ctypes.data, lo.ctypes.data, hi.ctypes.data))
    return _proposal_dict(ids, mean, chol, lo, hi, scale, prior_flags)


def fisher_proposal(ctx, theta0, sampled, scale=1.5, box_sigmas=10.0, chi_max=0.99, dmin=10.0, dmax=1000.0,
                    prior_flags=0):
    """The Gaussian proposal in the Fisher metric at theta0 (11 slots) over the sampled
    slots, with the slots the context marginalises projected out (mbis_fisher_proposal)."""
    th, pth = _host(theta0, np.float64)
    ids, pid = _host(sampled, np.int32)
    P = len(ids)
    mean, chol, lo, hi = np.zeros(P), np.zeros((P, P)), np.zeros(P), np.zeros(P)
    o = ProposalOptions(scale, box_sigmas, chi_max, dmin, dmax)
    _check(_lib.mbis_fisher_proposal(ctx, pth, P, pid, C.byref(o), mean.ctypes.data, chol.ctypes.data, lo.ctypes.data,
                                     hi.ctypes.data), ctx)
    return _proposal_dict(ids, mean, chol, lo, hi, scale, prior_flags)


# ------------------------------------------------------------------------------- tiled proposal
class TilingSpace(C.Structure):
    _fields_ = [("x_lo", C.c_double), ("x_hi", C.c_double), ("mc_period", C.c_double), ("mc_base", C.c_double),
                ("q_lo", C.c_double), ("q_hi", C.c_double), ("chi1", C.c_double), ("chi2", C.c_double)]


def _tcheck(status, t):
    if status != MBIS_OK:
        msg = _lib.mbis_tiling_last_error(t)
        raise MbisError(status, msg.decode() if msg else "")


def mbis_tiling_create(f_lo, df, n_bins, psd, x_lo, x_hi, mc_period, mc_base, q_lo, q_hi, chi1=0.0, chi2=0.0):
    grid = FreqGrid(f_lo, df, n_bins)
    psd_a, psd_p = _host(psd, np.float64)
    sp = TilingSpace(x_lo, x_hi, mc_period, mc_base, q_lo, q_hi, chi1, chi2)
    out = C.c_void_p()
    _tcheck(_lib.mbis_tiling_create(C.byref(grid), psd_p, C.byref(sp), C.byref(out)), None)
    return out.value


def mbis_tiling_destroy(t):
    _lib.mbis_tiling_destroy(t)


def mbis_tiling_bank(t, cand, min_match, stop_after, max_templates):
    """Stochastic placement over host candidates [2][n]; returns (n_templates, n_used)."""
    cand = np.ascontiguousarray(np.asarray(cand, dtype=np.float64).reshape(2, -1))
    nt, nu = C.c_int32(), C.c_int64()
    _tcheck(_lib.mbis_tiling_bank(t, cand.shape[1], cand.ctypes.data, min_match, stop_after, max_templates,
                                  C.byref(nt), C.byref(nu)), t)
    return nt.value, nu.value


def mbis_tiling_templates(t):
    """(coords [2][T], physical [2][T], candidate index [T]) of the bank."""
    nt = C.c_int32()
    _tcheck(_lib.mbis_tiling_templates(t, C.byref(nt), None, None, None), t)
    T = nt.value
    coords, phys, idx = np.zeros((2, T)), np.zeros((2, T)), np.zeros(T, dtype=np.int32)
    _tcheck(_lib.mbis_tiling_templates(t, C.byref(nt), coords.ctypes.data, phys.ctypes.data, idx.ctypes.data), t)
    return coords, phys, idx


def mbis_tiling_match(t, n, a, b, out, stream=None):
    _tcheck(_lib.mbis_tiling_match(t, n, _dev(a), _dev(b), _dev(out), _stream(stream)), t)


def mbis_tiling_assign(t, n, pts, tile, match=None, stream=None):
    _tcheck(_lib.mbis_tiling_assign(t, n, _dev(pts), _dev(tile), _dev(match), _stream(stream)), t)


def mbis_tiling_set_pool(t, n, pts, stream=None):
    _tcheck(_lib.mbis_tiling_set_pool(t, n, _dev(pts), _stream(stream)), t)


def mbis_tiling_pool(t, T, tile_of=None, members=None, stream=None):
    """Pool counts per tile (host int64 [T]); optionally copies the tile indices and member
    lists into device buffers."""
    counts = np.zeros(T, dtype=np.int64)
    _tcheck(_lib.mbis_tiling_pool(t, counts.ctypes.data, _dev(tile_of), _dev(members), _stream(stream)), t)
    return counts


def mbis_tiling_set_loglike(t, loglike_tpl, stream=None):
    _tcheck(_lib.mbis_tiling_set_loglike(t, _dev(loglike_tpl), _stream(stream)), t)


def mbis_tiling_draw(t, seed, ctr0, n, theta, log_q, log_prior, coords=None, pool_index=None, stream=None):
    _tcheck(_lib.mbis_tiling_draw(t, seed, ctr0, n, _dev(coords), _dev(theta), _dev(log_q), _dev(log_prior),
                                  _dev(pool_index), _stream(stream)), t)


# ------------------------------------------------------------------------------- P-P test
def mbis_credible_levels(n, theta, weights, ref, levels, stream=None):
    """Weighted fraction below ref [P] (host) of the samples theta [P][n] (device), into
    levels [P] (device)."""
    r, pr = _host(ref, np.float64)
    _check(_lib.mbis_credible_levels(n, len(r), _dev(theta), _dev(weights), pr, _dev(levels), _stream(stream)))


# ------------------------------------------------------------------------------- relative binning
def mbis_rb_setup(ctx, theta0, edges):
    t0, pt = _host(theta0, np.float64)
    e, pe = _host(edges, np.int32)
    _check(_lib.mbis_rb_setup(ctx, pt, len(e) - 1, pe), ctx)


def mbis_rb_loglike(ctx, n, theta, loglike, stream=None):
    _check(_lib.mbis_rb_loglike(ctx, n, _dev(theta), _dev(loglike), _stream(stream)), ctx)


def mbis_rb_use(ctx, on=True):
    """Route mbis_loglike and the ESS loop through the relative-binning likelihood (on) or
    back to the exact one."""
    _check(_lib.mbis_rb_use(ctx, 1 if on else 0), ctx)


def mbis_rb_edges(ctx, theta0, n_sigma, eps_rad, max_bins=65536):
    """Bin edges (int32 array of n_rb + 1) for relative binning about theta0."""
    t0, pt = _host(theta0, np.float64)
    edges = np.zeros(max_bins + 1, dtype=np.int32)
    nrb = C.c_int32()
    _check(_lib.mbis_rb_edges(ctx, pt, n_sigma, eps_rad, max_bins, edges.ctypes.data, C.byref(nrb)), ctx)
    return edges[:nrb.value + 1].copy()
