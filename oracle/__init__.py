"""Plain FP64 CPU oracle for metric-based importance sampling (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never imports it, and it imports nothing of
the product: the two share no code.  The arithmetic lives in ``mbis_oracle.c`` (plain C,
double precision, literal per-sample / per-detector / per-bin loops); this module only
builds that file and marshals numpy arrays into it.

Parameter slots of a full sample (shared interface numbering, also documented in the
C-ABI header of the product):
    0 Mc (detector-frame chirp mass, Msun)   1 q = m1/m2 >= 1   2 chi1z   3 chi2z
    4 RA (rad)  5 dec (rad)  6 psi (rad)  7 iota (rad)  8 d_L (Mpc)  9 t_c (s)  10 phi_c (rad)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mbis_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC = range(11)
NPAR = 11
MARG_PHASE, MARG_DISTANCE, MARG_TIME = 1, 2, 4
PRIOR_M1M2 = 1


def build(force: bool = False) -> str:
    """Compile ``mbis_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC) or not _native(LIB):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11",
               "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def _native(path):
    import platform
    import struct
    want = {"x86_64": 62, "amd64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine().lower())
    with open(path, "rb") as f:
        head = f.read(20)
    return head[:4] == b"\x7fELF" and (want is None or struct.unpack("<H", head[18:20])[0] == want)


class _Complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Event(C.Structure):
    _fields_ = [
        ("n_det", C.c_int32), ("n_bins", C.c_int32),
        ("f_lo", C.c_double), ("df", C.c_double),
        ("strain", C.c_void_p), ("psd", C.c_void_p),
        ("vertex", C.c_void_p), ("xarm", C.c_void_p), ("yarm", C.c_void_p),
        ("gmst", C.c_double),
        ("marg", C.c_uint32), ("n_tshift", C.c_int32), ("dt_shift", C.c_double),
        ("dmin", C.c_double), ("dmax", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, u32, u64, i32, p = C.c_double, C.c_int64, C.c_uint32, C.c_uint64, C.c_int32, C.c_void_p
        sig = {
            "or_philox4x32_10": (None, [p, p, p]),
            "or_box_muller": (None, [u32, u32, p, p]),
            "or_sample_normals": (None, [u64, u64, i32, p]),
            "or_psd_aligo": (d, [d]),
            "or_component_masses": (None, [d, d, p, p]),
            "or_mass_jacobian": (d, [d, d]),
            "or_pn_bracket": (d, [d, d, d, d, d]),
            "or_taylorf2_phase": (d, [d, p]),
            "or_f_isco": (d, [d, d]),
            "or_amplitude": (d, [d, d]),
            "or_polarisations": (None, [d, p, p, p]),
            "or_antenna": (None, [p, p, d, d, d, d, p, p]),
            "or_time_delay": (d, [p, d, d, d]),
            "or_detector_strain": (_Complex, [p, C.c_int, d, p]),
            "or_log_i0": (d, [d]),
            "or_distance_marginal": (d, [d, d, d, d]),
            "or_loglike": (d, [p, p]),
            "or_loglike_batch": (None, [p, i64, p, p]),
            "or_overlaps": (None, [p, p, p, p, p]),
            "or_make_strain": (None, [p, p, u64, C.c_int, p]),
            "or_optimal_snr2": (d, [p, p]),
            "or_fisher": (None, [p, p, i32, p, p, p]),
            "or_mass_prior_volume": (d, [d, d, d, d]),
            "or_log_prior": (d, [i32, p, p, p, u32, p]),
            "or_draw": (None, [u64, u64, i64, i32, p, p, p, d, p, p]),
            "or_reduce": (None, [i64, p, p, p, p, p]),
            "or_weighted_moments": (None, [i64, i32, p, p, p, p, p, p]),
            "or_tiling_physical": (None, [p, d, d, p, p]),
            "or_tiling_waveform": (i32, [p, d, d, p]),
            "or_tiling_overlap": (d, [i32, p, p]),
            "or_tiling_match": (d, [p, d, d, d, d]),
            "or_tiling_bank": (i32, [p, i64, p, d, i64, i32, p, p, p]),
            "or_tiling_assign": (None, [p, i64, p, i32, p, p, p, p]),
            "or_tiling_lists": (None, [i64, p, i32, p, p, p]),
            "or_tiling_mixture": (d, [i32, p, p, p]),
            "or_tiling_draw": (None, [u64, u64, i64, i32, p, d, p, p, p, p, i64, p, p, p]),
            "or_credible_levels": (None, [i64, i32, p, p, p, p]),
            "or_rb_loglike": (d, [p, p, i32, p, p]),
            "or_rb_loglike_batch": (None, [p, p, i32, p, i64, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------------------------------
class OracleEvent:
    """An event (data, PSD, detectors, options) held in memory the C oracle can read."""

    def __init__(self, f_lo, df, n_bins, psd, vertex, xarm, yarm, gmst=0.0, strain=None, marg=MARG_PHASE,
                 n_tshift=128, dt_shift=1e-4, dmin=10.0, dmax=1000.0):
        self.psd = _f64(psd).reshape(-1, n_bins)
        n_det = self.psd.shape[0]
        self.vertex = _f64(vertex).reshape(n_det, 3)
        self.xarm = _f64(xarm).reshape(n_det, 3)
        self.yarm = _f64(yarm).reshape(n_det, 3)
        self.strain = np.zeros((n_det, n_bins, 2)) if strain is None else _f64(strain).reshape(n_det, n_bins, 2)
        self.s = Event(n_det, n_bins, f_lo, df, _ptr(self.strain), _ptr(self.psd), _ptr(self.vertex),
                       _ptr(self.xarm), _ptr(self.yarm), gmst, marg, n_tshift, dt_shift, dmin, dmax)

    @property
    def n_det(self):
        return self.s.n_det

    @property
    def n_bins(self):
        return self.s.n_bins

    def freqs(self):
        return self.s.f_lo + np.arange(self.s.n_bins) * self.s.df

    def set_strain(self, strain):
        self.strain[...] = np.asarray(strain, dtype=np.float64).reshape(self.strain.shape)

    def with_marg(self, marg, **kw):
        ev = OracleEvent(self.s.f_lo, self.s.df, self.s.n_bins, self.psd, self.vertex, self.xarm, self.yarm,
                         self.s.gmst, self.strain, marg, kw.get("n_tshift", self.s.n_tshift),
                         kw.get("dt_shift", self.s.dt_shift), kw.get("dmin", self.s.dmin), kw.get("dmax", self.s.dmax))
        return ev


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def box_muller(a, b):
    z0, z1 = C.c_double(), C.c_double()
    lib().or_box_muller(a, b, C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def sample_normals(seed, g, P):
    z = np.zeros(P)
    lib().or_sample_normals(seed, g, P, _ptr(z))
    return z


def psd_aligo(f):
    return np.array([lib().or_psd_aligo(float(x)) for x in np.atleast_1d(f)])


def component_masses(mc, q):
    a, b = C.c_double(), C.c_double()
    lib().or_component_masses(mc, q, C.byref(a), C.byref(b))
    return a.value, b.value


def mass_jacobian(mc, q):
    return lib().or_mass_jacobian(mc, q)


def pn_bracket(v, m1, m2, chi1, chi2):
    return lib().or_pn_bracket(v, m1, m2, chi1, chi2)


def taylorf2_phase(f, par):
    par = _f64(par)
    return np.array([lib().or_taylorf2_phase(float(x), _ptr(par)) for x in np.atleast_1d(f)])


def f_isco(mc, q):
    return lib().or_f_isco(mc, q)


def amplitude(mc, dl):
    return lib().or_amplitude(mc, dl)


def polarisations(f, par):
    par = _f64(par)
    fs = np.atleast_1d(np.asarray(f, dtype=np.float64))
    hp = np.zeros(len(fs), dtype=np.complex128)
    hc = np.zeros(len(fs), dtype=np.complex128)
    a, b = np.zeros(2), np.zeros(2)
    for i, x in enumerate(fs):
        lib().or_polarisations(float(x), _ptr(par), _ptr(a), _ptr(b))
        hp[i] = a[0] + 1j * a[1]
        hc[i] = b[0] + 1j * b[1]
    return hp, hc


def antenna(xarm, yarm, ra, dec, psi, gmst):
    x, y = _f64(xarm), _f64(yarm)
    fp, fc = C.c_double(), C.c_double()
    lib().or_antenna(_ptr(x), _ptr(y), ra, dec, psi, gmst, C.byref(fp), C.byref(fc))
    return fp.value, fc.value


def time_delay(vertex, ra, dec, gmst):
    v = _f64(vertex)
    return lib().or_time_delay(_ptr(v), ra, dec, gmst)


def detector_strain(ev: OracleEvent, d, f, par):
    par = _f64(par)
    out = []
    for x in np.atleast_1d(f):
        r = lib().or_detector_strain(C.byref(ev.s), d, float(x), _ptr(par))
        out.append(r.re + 1j * r.im)
    return np.array(out)


def log_i0(x):
    return np.array([lib().or_log_i0(float(v)) for v in np.atleast_1d(x)])


def distance_marginal(z1, h1, dmin, dmax):
    return lib().or_distance_marginal(z1, h1, dmin, dmax)


def loglike(ev: OracleEvent, par):
    par = _f64(par)
    return lib().or_loglike(C.byref(ev.s), _ptr(par))


def loglike_batch(ev: OracleEvent, pars):
    pars = _f64(pars).reshape(-1, NPAR)
    out = np.zeros(len(pars))
    lib().or_loglike_batch(C.byref(ev.s), len(pars), _ptr(pars), _ptr(out))
    return out


def overlaps(ev: OracleEvent, par):
    par = _f64(par)
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().or_overlaps(C.byref(ev.s), _ptr(par), C.byref(a), C.byref(b), C.byref(c))
    return a.value + 1j * b.value, c.value


def make_strain(ev: OracleEvent, par, noise_seed=0, add_noise=False):
    par = _f64(par)
    out = np.zeros((ev.n_det, ev.n_bins, 2))
    lib().or_make_strain(C.byref(ev.s), _ptr(par), noise_seed, int(bool(add_noise)), _ptr(out))
    return out


def optimal_snr2(ev: OracleEvent, par):
    par = _f64(par)
    return lib().or_optimal_snr2(C.byref(ev.s), _ptr(par))


def fisher(ev: OracleEvent, par, ids, steps):
    par = _f64(par)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    steps = _f64(steps)
    P = len(ids)
    g = np.zeros((P, P))
    lib().or_fisher(C.byref(ev.s), _ptr(par), P, _ptr(ids), _ptr(steps), _ptr(g))
    return g


def mass_prior_volume(mc_lo, mc_hi, q_lo, q_hi):
    return lib().or_mass_prior_volume(mc_lo, mc_hi, q_lo, q_hi)


def log_prior(ids, lo, hi, flags, theta):
    """theta: P x n (SoA) -> n log prior values"""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    lo, hi = _f64(lo), _f64(hi)
    th = _f64(theta)
    P = len(ids)
    th = th.reshape(P, -1)
    out = np.empty(th.shape[1])
    col = np.empty(P)
    for i in range(th.shape[1]):
        col[:] = th[:, i]
        out[i] = lib().or_log_prior(P, _ptr(ids), _ptr(lo), _ptr(hi), flags, _ptr(col))
    return out


def draw(seed, ctr0, n, ids, mean, chol, scale):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    mean, chol = _f64(mean), _f64(chol)
    P = len(ids)
    theta = np.zeros((P, n))
    logq = np.zeros(n)
    lib().or_draw(seed, ctr0, n, P, _ptr(ids), _ptr(mean), _ptr(chol), scale, _ptr(theta), _ptr(logq))
    return theta, logq


def reduce(loglike, logp, logq, want_weights=False):
    ll, lp, lq = _f64(loglike), _f64(logp), _f64(logq)
    n = len(ll)
    w = np.zeros(n) if want_weights else None
    out = np.zeros(6)
    lib().or_reduce(n, _ptr(ll), _ptr(lp), _ptr(lq), _ptr(w) if w is not None else None, _ptr(out))
    res = dict(ess=out[0], log_z=out[1], max_logw=out[2], n=int(out[3]), s1=out[4], s2=out[5])
    if want_weights:
        res["weights"] = w
    return res


def weighted_moments(ids, theta, weights, ref):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    th, w, r = _f64(theta), _f64(weights), _f64(ref)
    P = len(ids)
    n = th.reshape(P, -1).shape[1]
    mean = np.zeros(P)
    cov = np.zeros((P, P))
    lib().or_weighted_moments(n, P, _ptr(ids), _ptr(th), _ptr(w), _ptr(r), _ptr(mean), _ptr(cov))
    return mean, cov


def full_params(ids, theta_cols, fixed):
    """Assemble n x 11 full parameter rows from sampled SoA columns and fixed values."""
    theta_cols = np.asarray(theta_cols, dtype=np.float64)
    n = theta_cols.shape[1]
    out = np.tile(np.asarray(fixed, dtype=np.float64), (n, 1))
    for p, i in enumerate(ids):
        out[:, i] = theta_cols[p]
    return out


# ------------------------------------------------------------------------------------------
# Tiled proposal (Sec. II; App. A)
class _TilingStruct(C.Structure):
    _fields_ = [("x_lo", C.c_double), ("x_hi", C.c_double), ("mc_period", C.c_double), ("mc_base", C.c_double),
                ("q_lo", C.c_double), ("q_hi", C.c_double), ("chi1", C.c_double), ("chi2", C.c_double),
                ("f_lo", C.c_double), ("df", C.c_double), ("n_bins", C.c_int32), ("psd", C.c_void_p)]


class Tiling:
    """The sampled space of the tiled proposal and the noise weighting of its match."""

    def __init__(self, f_lo, df, n_bins, psd, x_lo, x_hi, mc_period, mc_base, q_lo, q_hi, chi1=0.0, chi2=0.0):
        self.psd = _f64(psd).reshape(-1)
        assert len(self.psd) == n_bins
        self.s = _TilingStruct(x_lo, x_hi, mc_period, mc_base, q_lo, q_hi, chi1, chi2, f_lo, df, n_bins,
                               self.psd.ctypes.data)

    @property
    def n_bins(self):
        return self.s.n_bins

    def physical(self, x, q):
        mc, qp = C.c_double(), C.c_double()
        lib().or_tiling_physical(C.byref(self.s), float(x), float(q), C.byref(mc), C.byref(qp))
        return mc.value, qp.value

    def waveform(self, x, q):
        u = np.zeros(self.n_bins, dtype=np.complex128)
        live = lib().or_tiling_waveform(C.byref(self.s), float(x), float(q), _ptr(u))
        return u, live

    def match(self, xa, qa, xb, qb):
        return lib().or_tiling_match(C.byref(self.s), float(xa), float(qa), float(xb), float(qb))

    def bank(self, cand, min_match, stop_after, max_templates):
        """Stochastic placement over the candidates [2][n]; returns (indices, n_used, margin)."""
        cand = np.ascontiguousarray(_f64(cand).reshape(2, -1))
        n = cand.shape[1]
        idx = np.zeros(max_templates, dtype=np.int32)
        used, margin = C.c_int64(), C.c_double()
        T = lib().or_tiling_bank(C.byref(self.s), n, _ptr(cand), min_match, stop_after, max_templates, _ptr(idx),
                                 C.byref(used), C.byref(margin))
        return idx[:T].copy(), used.value, margin.value

    def assign(self, pts, templates):
        """Best template of each point [2][n] among templates [2][T]: (tile, match, runner-up)."""
        pts = np.ascontiguousarray(_f64(pts).reshape(2, -1))
        tpl = np.ascontiguousarray(_f64(templates).reshape(2, -1))
        n, T = pts.shape[1], tpl.shape[1]
        tile = np.zeros(n, dtype=np.int32)
        match, second = np.zeros(n), np.zeros(n)
        lib().or_tiling_assign(C.byref(self.s), n, _ptr(pts), T, _ptr(tpl), _ptr(tile), _ptr(match), _ptr(second))
        return tile, match, second


def tiling_lists(tile, T):
    tile = np.ascontiguousarray(tile, dtype=np.int32)
    n = len(tile)
    count, offset = np.zeros(T, dtype=np.int64), np.zeros(T, dtype=np.int64)
    members = np.zeros(max(n, 1), dtype=np.int64)
    lib().or_tiling_lists(n, _ptr(tile), T, _ptr(count), _ptr(offset), _ptr(members))
    return count, offset, members[:int(count.sum())]


def tiling_mixture(count, loglike_tpl):
    count = np.ascontiguousarray(count, dtype=np.int64)
    ll = _f64(loglike_tpl)
    c = np.zeros(len(count))
    m = lib().or_tiling_mixture(len(count), _ptr(count), _ptr(ll), _ptr(c))
    return c, m


def tiling_draw(seed, ctr0, n, c, m, loglike_tpl, count, offset, members, n_pool):
    """Draws of the tiled mixture: (pool index, tile, ln g - ln pi) per draw."""
    c, ll = _f64(c), _f64(loglike_tpl)
    count = np.ascontiguousarray(count, dtype=np.int64)
    offset = np.ascontiguousarray(offset, dtype=np.int64)
    members = np.ascontiguousarray(members, dtype=np.int64)
    idx, tile, lr = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int32), np.zeros(n)
    lib().or_tiling_draw(seed, ctr0, n, len(c), _ptr(c), m, _ptr(ll), _ptr(count), _ptr(offset), _ptr(members),
                         n_pool, _ptr(idx), _ptr(tile), _ptr(lr))
    return idx, tile, lr


def credible_levels(theta, weights, ref):
    """Weighted fraction of the samples [P][n] below ref [P] per slot (ties count half)."""
    th, w, r = _f64(theta), _f64(weights), _f64(ref)
    P = len(r)
    n = th.reshape(P, -1).shape[1]
    out = np.zeros(P)
    lib().or_credible_levels(n, P, _ptr(th), _ptr(w), _ptr(r), _ptr(out))
    return out


def rb_loglike_batch(ev: OracleEvent, par0, edges, pars):
    """Relative-binning log-likelihood ratios of n x 11 parameter rows about the fiducial
    par0 with bin edges (bin indices, edges[0] = 0, edges[-1] = n_bins)."""
    pars = _f64(pars).reshape(-1, NPAR)
    p0 = _f64(par0)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    out = np.zeros(len(pars))
    lib().or_rb_loglike_batch(C.byref(ev.s), _ptr(p0), len(e) - 1, _ptr(e), len(pars), _ptr(pars), _ptr(out))
    return out
