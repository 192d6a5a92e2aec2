"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds no arithmetic of the method: it only states the workload recipes
(frequency grids, detector networks, sampled-parameter sets, options) and draws the
population parameters of synthetic events from a seeded numpy generator.  Waveforms,
noise, PSDs, likelihoods, proposals and weights are computed by each side on its own.

The paper simulates its populations (Sec. III A) and runs no public dataset through
this path; these recipes stand in for its BNS and BBH populations with the shapes the
benchmark configurations name.

Parameter slots (the numbering of the C-ABI and of the oracle):
    0 Mc  1 q  2 chi1z  3 chi2z  4 RA  5 dec  6 psi  7 iota  8 d_L  9 t_c  10 phi_c
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC = range(11)
NPAR = 11
PARAM_NAMES = ["mc", "q", "chi1", "chi2", "ra", "dec", "psi", "iota", "dl", "tc", "phic"]
MARG_PHASE, MARG_DISTANCE, MARG_TIME = 1, 2, 4
PRIOR_M1M2 = 1

POPULATION_SEED = 0x241005190

# Detector geometry: vertex (Earth-centred Earth-fixed, metres) and unit arm vectors.
# Anderson, Brady, Creighton & Flanagan (2001), Table I (LIGO Hanford, LIGO Livingston,
# Virgo).  Geometry is input data to both sides of every comparison.
DETECTORS = {
    "H1": dict(vertex=(-2161414.92636, -3834695.17889, 4600350.22664),
               xarm=(-0.22389266154, 0.79983062746, 0.55690487831),
               yarm=(-0.91397818574, 0.02609403989, -0.40492342125)),
    "L1": dict(vertex=(-74276.0447238, -5496283.71971, 3224257.01744),
               xarm=(-0.95457412153, -0.14158077340, -0.26218911324),
               yarm=(0.29774156894, -0.48791033647, -0.82054461286)),
    "V1": dict(vertex=(4546374.099, 842989.6976, 4378576.963),
               xarm=(-0.70045821479, 0.20848948619, 0.68256166277),
               yarm=(-0.05379255368, -0.96908180549, 0.24080451708)),
}


def network(names):
    """(vertex, xarm, yarm) arrays, each n_det x 3, for a list of detector names."""
    v = np.array([DETECTORS[n]["vertex"] for n in names], dtype=np.float64)
    x = np.array([DETECTORS[n]["xarm"] for n in names], dtype=np.float64)
    y = np.array([DETECTORS[n]["yarm"] for n in names], dtype=np.float64)
    return v, x, y


def n_bins_for(f_lo, f_hi, df):
    """Number of grid points f_lo + k df, k = 0..n-1, with both ends included."""
    return int(round((f_hi - f_lo) / df)) + 1


@dataclass
class EventSpec:
    """One synthetic event: true parameters (m1, m2 in Msun, and the rest by slot), the
    target network SNR, the noise seed (None: zero noise) and the proposal seed."""
    m1: float
    m2: float
    params: dict            # slot name -> value for chi1, chi2, ra, dec, psi, iota, tc, phic
    gmst: float
    snr: float
    noise_seed: int | None
    draw_seed: int


@dataclass
class Workload:
    name: str
    detectors: list
    f_lo: float
    f_hi: float
    df: float
    sampled: list           # parameter slots drawn from the proposal
    marg: int               # MARG_* bits
    n_samples: int          # proposal samples per event
    precision: str          # "fp64" or "mixed"
    complex_dtype: str      # strain storage: "c128" or "c64"
    scale: float            # proposal width scale s
    prior_flags: int
    chi_max: float
    events: list = field(default_factory=list)
    n_tshift: int = 128
    dt_shift: float = 1e-4
    dmin: float = 10.0
    dmax: float = 1000.0
    box_sigmas: float = 10.0  # half-width of the (Mc, q, t_c) prior box in proposal sigmas

    @property
    def n_bins(self):
        return n_bins_for(self.f_lo, self.f_hi, self.df)

    @property
    def n_det(self):
        return len(self.detectors)


def _isotropic(rng):
    ra = rng.uniform(0.0, 2 * math.pi)
    dec = math.asin(rng.uniform(-1.0, 1.0))
    psi = rng.uniform(0.0, math.pi)
    iota = math.acos(rng.uniform(-1.0, 1.0))
    return ra, dec, psi, iota


def tiny(n_samples=4096):
    """One zero-noise event, H1+L1, 20-512 Hz at 0.25 Hz (1969 bins, complex128), 4
    sampled intrinsics (Mc, q, chi1, chi2), phase marginalised, FP64."""
    ev = EventSpec(m1=30.0, m2=25.0,
                   params=dict(chi1=0.3, chi2=-0.1, ra=1.0, dec=0.5, psi=0.3, iota=0.4, tc=0.0, phic=0.0),
                   gmst=0.0, snr=15.0, noise_seed=None, draw_seed=POPULATION_SEED ^ 0x11)
    return Workload("tiny", ["H1", "L1"], 20.0, 512.0, 0.25, [MC, Q, CHI1, CHI2], MARG_PHASE, n_samples,
                    "fp64", "c128", 1.0, 0, 0.99, [ev])


def bns_population(n_events=256, n_samples=1 << 20, seed=POPULATION_SEED):
    """Aligned-spin BNS population: m1, m2 ~ U[1.1, 2.0] (sorted), chi ~ U[-0.05, 0.05],
    isotropic sky and orientation, SNR ~ U[10, 30], coloured Gaussian noise; H1+L1,
    20-1024 Hz at 1/128 Hz (128,513 bins, complex64); sampled (Mc, q, chi1, chi2, t_c);
    phase and distance marginalised; prior flat in component masses."""
    rng = np.random.Generator(np.random.PCG64(seed))
    events = []
    for e in range(n_events):
        m = np.sort(rng.uniform(1.1, 2.0, size=2))[::-1]
        chi = rng.uniform(-0.05, 0.05, size=2)
        ra, dec, psi, iota = _isotropic(rng)
        gmst = rng.uniform(0.0, 2 * math.pi)
        phic = rng.uniform(0.0, 2 * math.pi)
        snr = rng.uniform(10.0, 30.0)
        events.append(EventSpec(float(m[0]), float(m[1]),
                                dict(chi1=float(chi[0]), chi2=float(chi[1]), ra=ra, dec=dec, psi=psi, iota=iota,
                                     tc=0.0, phic=phic),
                                gmst, snr, noise_seed=(seed << 8) + 2 * e + 1, draw_seed=(seed << 8) + 2 * e + 2))
    return Workload("bns_population", ["H1", "L1"], 20.0, 1024.0, 1.0 / 128, [MC, Q, CHI1, CHI2, TC],
                    MARG_PHASE | MARG_DISTANCE, n_samples, "mixed", "c64", 1.5, PRIOR_M1M2, 0.05, events)


def bbh_population(n_events=128, n_samples=1 << 18, seed=POPULATION_SEED + 3):
    """Aligned-spin BBH with full extrinsics: m1, m2 ~ U[10, 80] (sorted),
    chi ~ U[-0.8, 0.8], isotropic, SNR ~ U[10, 40]; H1+L1+V1, 20-1024 Hz at 1/8 Hz
    (8033 bins); all 11 parameters sampled except d_L... (d_L sampled too: 11 params);
    time marginalised over 128 shifts of 0.1 ms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    events = []
    for e in range(n_events):
        m = np.sort(rng.uniform(10.0, 80.0, size=2))[::-1]
        chi = rng.uniform(-0.8, 0.8, size=2)
        ra, dec, psi, iota = _isotropic(rng)
        gmst = rng.uniform(0.0, 2 * math.pi)
        phic = rng.uniform(0.0, 2 * math.pi)
        snr = rng.uniform(10.0, 40.0)
        events.append(EventSpec(float(m[0]), float(m[1]),
                                dict(chi1=float(chi[0]), chi2=float(chi[1]), ra=ra, dec=dec, psi=psi, iota=iota,
                                     tc=0.0, phic=phic),
                                gmst, snr, noise_seed=(seed << 8) + 2 * e + 1, draw_seed=(seed << 8) + 2 * e + 2))
    return Workload("bbh_population", ["H1", "L1", "V1"], 20.0, 1024.0, 1.0 / 8,
                    [MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC], MARG_TIME, n_samples, "mixed", "c64",
                    1.5, PRIOR_M1M2, 0.8, events)


UNEVEN_DF = [1.0 / 4, 1.0 / 8, 1.0 / 16, 1.0 / 32, 1.0 / 64, 1.0 / 128]


def uneven_batch(n_events=64, seed=POPULATION_SEED + 4):
    """Events of uneven size for one persistent launch, alternating two families:

    * heavy (the plain-method family): m1, m2 ~ U[20, 40] (sorted), chi ~ U[-0.5, 0.5],
      20-512 Hz, sampled (Mc, q, chi1, chi2), phase marginalised, SNR ~ U[10, 30];
    * BNS (the population family): m1, m2 ~ U[1.1, 2.0], chi ~ U[-0.05, 0.05], 20-1024 Hz,
      sampled (Mc, q, chi1, chi2, t_c), phase and distance marginalised, SNR ~ U[10, 30];

    each with df drawn from {1/4, ..., 1/128} Hz (1,969 to 128,513 bins), H1+L1 or
    H1+L1+V1 (fixed extrinsics), 2^14 .. 2^20 samples, coloured Gaussian noise, complex64
    data, mixed precision.  Returns one single-event Workload per event."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for e in range(n_events):
        bns = e % 2 == 1
        df = UNEVEN_DF[int(rng.integers(0, len(UNEVEN_DF)))]
        dets = ["H1", "L1", "V1"] if rng.uniform() < 0.5 else ["H1", "L1"]
        n_samples = 1 << int(rng.integers(14, 21))
        if bns:
            m = np.sort(rng.uniform(1.1, 2.0, size=2))[::-1]
            chi = rng.uniform(-0.05, 0.05, size=2)
        else:
            m = np.sort(rng.uniform(20.0, 40.0, size=2))[::-1]
            chi = rng.uniform(-0.5, 0.5, size=2)
        ra, dec, psi, iota = _isotropic(rng)
        gmst = rng.uniform(0.0, 2 * math.pi)
        phic = rng.uniform(0.0, 2 * math.pi)
        snr = rng.uniform(10.0, 30.0)
        spec = EventSpec(float(m[0]), float(m[1]),
                         dict(chi1=float(chi[0]), chi2=float(chi[1]), ra=ra, dec=dec, psi=psi, iota=iota, tc=0.0,
                              phic=phic),
                         gmst, snr, noise_seed=(seed << 8) + 2 * e + 1, draw_seed=(seed << 8) + 2 * e + 2)
        if bns:
            w = Workload(f"uneven_{e}_bns", dets, 20.0, 1024.0, df, [MC, Q, CHI1, CHI2, TC],
                         MARG_PHASE | MARG_DISTANCE, n_samples, "mixed", "c64", 1.5, PRIOR_M1M2, 0.05, [spec])
        else:
            w = Workload(f"uneven_{e}_heavy", dets, 20.0, 512.0, df, [MC, Q, CHI1, CHI2], MARG_PHASE, n_samples,
                         "mixed", "c64", 1.5, 0, 0.5, [spec])
        out.append(w)
    return out


@dataclass
class TiledDemo:
    """The two-parameter demonstration of the tiled proposal (App. A): one BBH event whose
    sampled coordinates are a cyclic chirp mass x (chirp mass mc_base + mod(x, mc_period),
    over two periods) and a mass ratio q over [1/q_max, q_max] (q and 1/q are the same
    binary), so the posterior has four modes.  Prior uniform in (x, q)."""
    workload: Workload       # the event: sampled slots (Mc, q) of the physical space
    x_lo: float
    x_hi: float
    mc_period: float
    mc_base: float
    q_lo: float
    q_hi: float
    min_match: float
    stop_after: int
    max_templates: int
    n_candidates: int
    candidate_seed: int
    n_pool: int
    pool_seed: int
    draw_seed: int


def tiled_demo(n_pool=1 << 22, snr=15.0, seed=POPULATION_SEED + 5):
    """Source at Mc = 25, q = 3.5 (m1 = 55.75, m2 = 15.93 Msun), zero spins, fixed sky and
    orientation, H1+L1, 20-128 Hz at 1/4 Hz (433 bins; every waveform of the space ends
    below 80 Hz), coloured Gaussian noise at network SNR 15, phase marginalised; x in [20, 28) with Mc = 24 + mod(x, 4), q in [1/6, 6]; bank
    at minimal match 0.996, stopping after 2000 consecutive rejections; a prior pool of
    2^22 points."""
    mc, q = 25.0, 3.5
    m1 = mc * (1.0 + q) ** 0.2 * q ** 0.4
    m2 = m1 / q
    spec = EventSpec(m1, m2, dict(chi1=0.0, chi2=0.0, ra=1.0, dec=0.5, psi=0.3, iota=0.4, tc=0.0, phic=0.0),
                     gmst=0.0, snr=snr, noise_seed=(seed << 8) + 1, draw_seed=(seed << 8) + 2)
    w = Workload("tiled_demo", ["H1", "L1"], 20.0, 128.0, 0.25, [MC, Q], MARG_PHASE, 1 << 16, "mixed", "c64",
                 1.0, 0, 0.0, [spec])
    return TiledDemo(w, 20.0, 28.0, 4.0, 24.0, 1.0 / 6.0, 6.0, 0.996, 2000, 4096, 1 << 17, (seed << 8) + 3,
                     n_pool, (seed << 8) + 4, (seed << 8) + 5)


def uniform_points(n, x_lo, x_hi, q_lo, q_hi, seed):
    """n points uniform in the box [x_lo, x_hi) x [q_lo, q_hi] as a [2][n] array (x row, q
    row): candidates of the template placement and the prior pool of the tiles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((2, n))
    out[0] = rng.uniform(x_lo, x_hi, n)
    out[1] = rng.uniform(q_lo, q_hi, n)
    return out


def tiled_population(demo: "TiledDemo", n_events, seed=POPULATION_SEED + 6):
    """Sources of the tiled demonstration space drawn from its prior (uniform in x and q),
    phase uniform in [0, 2 pi), a common luminosity distance (the one giving network SNR
    15 to the demonstration source), noise and draw seeds: the P-P population."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(demo.x_lo, demo.x_hi, n_events)
    q = rng.uniform(demo.q_lo, demo.q_hi, n_events)
    phic = rng.uniform(0.0, 2 * math.pi, n_events)
    return [dict(x=float(x[e]), q=float(q[e]), phic=float(phic[e]), noise_seed=(seed << 8) + 2 * e + 1,
                 draw_seed=(seed << 8) + 2 * e + 2) for e in range(n_events)]


PP_BOX = {MC: (1.1, 1.5), Q: (1.0, 1.6), TC: (-5e-4, 5e-4)}
PP_MASS_SQUARE = (1.0, 2.2)       # component masses drawn in this square, then cut to the box


def bns_pp_population(n_events=64, seed=POPULATION_SEED + 7):
    """BNS sources drawn from the fixed prior that their analysis uses, for the P-P test:
    flat in (m1, m2) inside Mc in [1.1, 1.5], q = m1/m2 in [1, 1.6] (by rejection from
    m ~ U[1.0, 2.2] sorted, a square that holds the whole box: m2 >= 1.004, m1 <= 2.19 there),
    chi ~ U[-0.05, 0.05], t_c ~ U[-0.5, 0.5] ms, isotropic sky and
    orientation, SNR ~ U[10, 30], coloured noise; H1+L1, 20-1024 Hz at 1/128 Hz; sampled
    (Mc, q, chi1, chi2, t_c); phase and distance marginalised.  The analysis box is PP_BOX."""
    rng = np.random.Generator(np.random.PCG64(seed))
    events = []
    for e in range(n_events):
        while True:
            m = np.sort(rng.uniform(*PP_MASS_SQUARE, size=2))[::-1]
            mc = (m[0] * m[1]) ** 0.6 / (m[0] + m[1]) ** 0.2
            if PP_BOX[MC][0] <= mc <= PP_BOX[MC][1] and m[0] / m[1] <= PP_BOX[Q][1]:
                break
        chi = rng.uniform(-0.05, 0.05, size=2)
        ra, dec, psi, iota = _isotropic(rng)
        gmst = rng.uniform(0.0, 2 * math.pi)
        phic = rng.uniform(0.0, 2 * math.pi)
        tc = rng.uniform(*PP_BOX[TC])
        snr = rng.uniform(10.0, 30.0)
        events.append(EventSpec(float(m[0]), float(m[1]),
                                dict(chi1=float(chi[0]), chi2=float(chi[1]), ra=ra, dec=dec, psi=psi, iota=iota,
                                     tc=tc, phic=phic),
                                gmst, snr, noise_seed=(seed << 8) + 2 * e + 1, draw_seed=(seed << 8) + 2 * e + 2))
    return Workload("bns_pp_population", ["H1", "L1"], 20.0, 1024.0, 1.0 / 128, [MC, Q, CHI1, CHI2, TC],
                    MARG_PHASE | MARG_DISTANCE, 1 << 18, "mixed", "c64", 1.5, PRIOR_M1M2, 0.05, events)


PP_BOX_BBH = {MC: (15.0, 30.0), Q: (1.0, 4.0), TC: (-1e-3, 1e-3)}
PP_MASS_SQUARE_BBH = (9.0, 75.0)


def bbh_pp_population(n_events=64, seed=POPULATION_SEED + 8):
    """BBH sources for the P-P test of the intrinsic parameters, drawn from the fixed prior
    their analysis uses: flat in (m1, m2) inside Mc in [15, 30], q = m1/m2 in [1, 4] (by
    rejection from m ~ U[9, 75] sorted, a square that holds the whole box: m2 >= 9.008,
    m1 <= 72.07 there), chi ~ U[-0.8, 0.8],
    t_c ~ U[-1, 1] ms, isotropic sky and orientation held fixed in the analysis, SNR ~
    U[10, 40], coloured noise; H1+L1+V1, 20-1024 Hz at 1/8 Hz; sampled (Mc, q, chi1, chi2,
    t_c); phase and distance marginalised.  The analysis box is PP_BOX_BBH."""
    rng = np.random.Generator(np.random.PCG64(seed))
    events = []
    for e in range(n_events):
        while True:
            m = np.sort(rng.uniform(*PP_MASS_SQUARE_BBH, size=2))[::-1]
            mc = (m[0] * m[1]) ** 0.6 / (m[0] + m[1]) ** 0.2
            if PP_BOX_BBH[MC][0] <= mc <= PP_BOX_BBH[MC][1] and m[0] / m[1] <= PP_BOX_BBH[Q][1]:
                break
        chi = rng.uniform(-0.8, 0.8, size=2)
        ra, dec, psi, iota = _isotropic(rng)
        gmst = rng.uniform(0.0, 2 * math.pi)
        phic = rng.uniform(0.0, 2 * math.pi)
        tc = rng.uniform(*PP_BOX_BBH[TC])
        snr = rng.uniform(10.0, 40.0)
        events.append(EventSpec(float(m[0]), float(m[1]),
                                dict(chi1=float(chi[0]), chi2=float(chi[1]), ra=ra, dec=dec, psi=psi, iota=iota,
                                     tc=tc, phic=phic),
                                gmst, snr, noise_seed=(seed << 8) + 2 * e + 1, draw_seed=(seed << 8) + 2 * e + 2))
    return Workload("bbh_pp_population", ["H1", "L1", "V1"], 20.0, 1024.0, 1.0 / 8, [MC, Q, CHI1, CHI2, TC],
                    MARG_PHASE | MARG_DISTANCE, 1 << 18, "mixed", "c64", 1.5, PRIOR_M1M2, 0.8, events)


def scaled(w: Workload, n_events=None, n_samples=None, f_hi=None):
    """A copy of a workload with fewer events, fewer samples or a shorter band (for the
    oracle-sized parity cases)."""
    import copy
    out = copy.deepcopy(w)
    if n_events is not None:
        out.events = out.events[:n_events]
    if n_samples is not None:
        out.n_samples = n_samples
    if f_hi is not None:
        out.f_hi = f_hi
    return out
