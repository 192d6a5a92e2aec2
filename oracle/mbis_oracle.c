/*
 * mbis_oracle.c -- plain FP64 reference of metric-based importance sampling for
 * compact-binary parameter estimation (Nitz, "Robust, Rapid, and Simple
 * Gravitational-wave Parameter Estimation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this file.  The product library never includes, links or
 * calls it, and this file includes nothing of the product: the two share no code.
 *
 * Every function evaluates its definition literally, in double precision, per sample,
 * per detector and per frequency bin: no tables, no anchors, no folded sums, no
 * reordering beyond what the definition states.  Each function names the passage it
 * follows.  Where the paper is silent (it prints no waveform, PSD, detector geometry,
 * prior or marginalisation formula), the reading taken is stated beside the code.
 *
 * Pins (tests that tie this file to something other than itself):
 *   philox / Box-Muller ........ published known-answer vectors; normal moments + KS
 *   PSD ........................ value at the knee frequency; positivity
 *   masses / Jacobian .......... round trip through an independent chirp-mass formula;
 *                                finite-difference determinant
 *   TaylorF2 non-spinning ...... series of -E'(v)/F(v) from the PN energy and flux
 *   TaylorF2 spin-orbit ........ 1.5, 2.5, 3 and 3.5PN terms re-derived from the
 *                                spin-orbit PN energy and flux, every mass ratio
 *   TaylorF2 spins, test mass .. every spin term at eta -> 0 re-derived from the Kerr
 *                                circular-orbit energy and the perturbative flux
 *   TaylorF2 1.5PN/2PN spins ... chi_s/chi_a form vs the (beta, sigma) form used here
 *   TaylorF2 3PN spin-spin ..... the per-body (kappa = 1) form; label swap
 *   amplitude .................. SPA of the quadrupole chirp; flat-PSD closed-form <h|h>
 *   antenna / delays ........... zenith, arm and bisector special cases; psi invariance;
 *                                baseline light-travel time; delay == shifted t_c
 *   log I0 ..................... scipy i0e and periodic-trapezoid quadrature
 *   marginalisations ........... brute force over phi_c, d_L and t_c of the
 *                                unmarginalised likelihood; scipy quad for distance
 *   draws / log g / prior ...... scipy multivariate normal; empirical moments;
 *                                prior normalises to one
 *   weights / ESS / log Z ...... equal weights, single weight, Gaussian target with
 *                                proposal == target (ESS = N, closed-form evidence)
 *   Fisher matrix .............. closed forms for ln d_L, phi_c and their cross term
 *   tiling match ............... the normalised overlap of the likelihood's inner product
 *                                of detector strains; the phase-projected Fisher metric
 *   bank / tiles ............... packing and covering invariants; brute-force argmax;
 *                                images of one binary share a tile
 *   mixture / draws ............ E_g[w] = mean prior likelihood exactly; equal weights
 *                                (ESS = n) when L is constant per tile; frequencies
 *   credible levels ............ order statistics of equal weights; mirror symmetry; the
 *                                Gaussian posterior of a linear model (normal CDF)
 *   relative binning ........... exact at the fiducial and with one frequency per bin;
 *                                second-order convergence in the bin width
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_TWO_PI 6.28318530717958647692
#define OR_T_SUN 4.925490947641267e-6  /* G M_sun / c^3 in s (IAU 2015 nominal) */
#define OR_MPC_M 3.0856775814913673e22 /* metres per megaparsec */
#define OR_C_MS 299792458.0            /* speed of light, m/s */
#define OR_EULER_GAMMA 0.57721566490153286061

/* parameter slots of a full 11-parameter sample */
enum { OR_MC = 0, OR_Q, OR_CHI1, OR_CHI2, OR_RA, OR_DEC, OR_PSI, OR_IOTA, OR_DL, OR_TC, OR_PHIC, OR_NPAR };
/* marginalisation modes */
enum { OR_MARG_PHASE = 1, OR_MARG_DISTANCE = 2, OR_MARG_TIME = 4 };
/* prior flags */
enum { OR_PRIOR_M1M2 = 1 };

typedef struct {
  int32_t n_det, n_bins;
  double f_lo, df;
  const double* strain; /* [n_det][n_bins][2]  (re, im) */
  const double* psd;    /* [n_det][n_bins]     one-sided PSD */
  const double* vertex; /* [n_det][3]  ECEF metres */
  const double* xarm;   /* [n_det][3]  unit vector */
  const double* yarm;   /* [n_det][3]  unit vector */
  double gmst;          /* Greenwich mean sidereal time at t_ref, rad */
  uint32_t marg;        /* OR_MARG_* */
  int32_t n_tshift;     /* time-marginalisation grid size J */
  double dt_shift;      /* grid spacing, s */
  double dmin, dmax;    /* distance prior range, Mpc */
} or_event;

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), written from
 * its published definition: 10 rounds of two 32x32->64 multiplies with Weyl key bumps. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in the open interval (0, 1) from one 32-bit word */
static double or_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Box-Muller: two independent standard normals from two uniforms */
void or_box_muller(uint32_t a, uint32_t b, double* z0, double* z1) {
  double u1 = or_uniform(a), u2 = or_uniform(b);
  double r = sqrt(-2.0 * log(u1));
  *z0 = r * cos(OR_TWO_PI * u2);
  *z1 = r * sin(OR_TWO_PI * u2);
}

/* P standard normals of proposal sample g: counter (lo g, hi g, 2, block), key = seed */
void or_sample_normals(uint64_t seed, uint64_t g, int32_t P, double* z) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t j = 0; 4 * j < P; ++j) {
    uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), 2u, (uint32_t)j}, w[4];
    or_philox4x32_10(ctr, key, w);
    double n[4];
    or_box_muller(w[0], w[1], &n[0], &n[1]);
    or_box_muller(w[2], w[3], &n[2], &n[3]);
    for (int i = 0; i < 4 && 4 * j + i < P; ++i) z[4 * j + i] = n[i];
  }
}

/* ------------------------------------------------------------------------------------ */
/* Frequency grid (Eq. 1 discretised): f_k = f_lo + k df for k = 0 .. n_bins-1, every bin
 * weighted by df (rectangle rule, no half weights at the ends). */
double or_freq(double f_lo, double df, int64_t k) { return f_lo + (double)k * df; }

/* Analytic aLIGO-like PSD fit (Ajith 2011), x = f / 215 Hz.  The paper says only
 * "sensitivity consistent with Advanced LIGO's third observing run" (Sec. III A). */
double or_psd_aligo(double f) {
  double x = f / 215.0, x2 = x * x;
  return 1e-49 * (pow(x, -4.14) - 5.0 / x2 + 111.0 * (1.0 - x2 + 0.5 * x2 * x2) / (1.0 + 0.5 * x2));
}

/* Component masses from chirp mass and mass ratio q = m1/m2 (the q > 1 convention of
 * App. A). */
void or_component_masses(double mc, double q, double* m1, double* m2) {
  *m1 = mc * pow(1.0 + q, 0.2) * pow(q, 0.4);
  *m2 = mc * pow(1.0 + q, 0.2) * pow(q, -0.6);
}

/* |d(m1, m2) / d(Mc, q)|: density of a prior flat in component masses, in (Mc, q) */
double or_mass_jacobian(double mc, double q) {
  double m1, m2;
  or_component_masses(mc, q, &m1, &m2);
  return m1 * m2 / (mc * q);
}

/* ------------------------------------------------------------------------------------ */
/* TaylorF2 phase (aligned spins, 3.5PN).  The paper models signals with IMRPhenom
 * families (Sec. III); this build uses the closed-form TaylorF2 inspiral instead.  The
 * coefficients follow Buonanno, Iyer, Ochsner, Pan & Sathyaprakash (2009) for the
 * non-spinning part and the chi_s/chi_a collection of Khan et al. (2016, App. B) for
 * the spin terms.  The 1.5PN and 2PN spin terms are written here in the (beta, sigma)
 * form so that a test can compare them with the chi_s/chi_a form.  Readings: the GW
 * phase convention h ~ exp(-i Psi); the 2.5PN log term is (1 + 3 ln v) with no v_lso;
 * phi_c is the GW phase; the spin-squared (tail) and spin-cubed 3.5PN terms and the
 * quadrupole-monopole (kappa != 1) terms are omitted.  The delta chi_a term of the 2.5PN
 * factor carries -140/9 eta: the sign that the spin-orbit energy and flux imply.
 *
 * Returns sum_n phi_n(v) v^n for n = 0..7, the bracket of
 *   Psi(f) = 2 pi f t_c - phi_c - pi/4 + 3 / (128 eta v^5) * bracket,  v = (pi M f)^(1/3). */
double or_pn_bracket(double v, double m1, double m2, double chi1, double chi2) {
  const double pi = OR_PI, pi2 = OR_PI * OR_PI;
  double M = m1 + m2, X1 = m1 / M, X2 = m2 / M, eta = X1 * X2;
  double delta = X1 - X2, chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
  double eta2 = eta * eta, eta3 = eta2 * eta;

  /* 1.5PN spin-orbit and 2PN spin-spin combinations */
  double beta = (chi1 * (113.0 * X1 * X1 + 75.0 * eta) + chi2 * (113.0 * X2 * X2 + 75.0 * eta)) / 12.0;
  double sigma = 79.0 / 8.0 * eta * chi1 * chi2 + 81.0 / 16.0 * (X1 * X1 * chi1 * chi1 + X2 * X2 * chi2 * chi2);

  double p0 = 1.0;
  double p1 = 0.0;
  double p2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
  double p3 = -16.0 * pi + 4.0 * beta;
  double p4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta2 - 10.0 * sigma;
  double p5 = (1.0 + 3.0 * log(v)) *
              (pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) +
               delta * (-732985.0 / 2268.0 - 140.0 / 9.0 * eta) * chia +
               (-732985.0 / 2268.0 + 24260.0 / 81.0 * eta + 340.0 / 9.0 * eta2) * chis);
  double p6 = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 -
              6848.0 / 21.0 * (OR_EULER_GAMMA + log(4.0 * v)) +
              (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) * eta + 76055.0 / 1728.0 * eta2 -
              127825.0 / 1296.0 * eta3 +
              pi * (2270.0 / 3.0 * delta * chia + (2270.0 / 3.0 - 520.0 * eta) * chis) +
              (75515.0 / 144.0 - 8225.0 / 18.0 * eta) * delta * chia * chis +
              (75515.0 / 288.0 - 263245.0 / 252.0 * eta - 480.0 * eta2) * chia * chia +
              (75515.0 / 288.0 - 232415.0 / 504.0 * eta + 1255.0 / 9.0 * eta2) * chis * chis;
  double p7 = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta2) +
              (-25150083775.0 / 3048192.0 + 10566655595.0 / 762048.0 * eta - 1042165.0 / 3024.0 * eta2 +
               5345.0 / 36.0 * eta3) * chis +
              delta * (-25150083775.0 / 3048192.0 + 26804935.0 / 6048.0 * eta - 1985.0 / 48.0 * eta2) * chia;

  double v2 = v * v, v3 = v2 * v, v4 = v3 * v, v5 = v4 * v, v6 = v5 * v, v7 = v6 * v;
  return p0 + p1 * v + p2 * v2 + p3 * v3 + p4 * v4 + p5 * v5 + p6 * v6 + p7 * v7;
}

/* GW phase Psi(f) in radians; par holds the 11 parameters. */
double or_taylorf2_phase(double f, const double* par) {
  double m1, m2;
  or_component_masses(par[OR_MC], par[OR_Q], &m1, &m2);
  double M = m1 + m2, eta = m1 * m2 / (M * M);
  double v = cbrt(OR_PI * M * OR_T_SUN * f);
  double bracket = or_pn_bracket(v, m1, m2, par[OR_CHI1], par[OR_CHI2]);
  return OR_TWO_PI * f * par[OR_TC] - par[OR_PHIC] - OR_PI / 4.0 + 3.0 / (128.0 * eta * pow(v, 5)) * bracket;
}

/* Termination: Schwarzschild ISCO of the total mass; bins with f >= f_isco are zero
 * (the paper's waveforms end on their own; a hard cut is this build's reading). */
double or_f_isco(double mc, double q) {
  double m1, m2;
  or_component_masses(mc, q, &m1, &m2);
  return 1.0 / (pow(6.0, 1.5) * OR_PI * (m1 + m2) * OR_T_SUN);
}

/* Amplitude of the f^(-7/6) inspiral: sqrt(5/24) pi^(-2/3) (Mc T_sun)^(5/6) / (d_L / c). */
double or_amplitude(double mc, double dl_mpc) {
  return sqrt(5.0 / 24.0) * pow(OR_PI, -2.0 / 3.0) * pow(mc * OR_T_SUN, 5.0 / 6.0) / (dl_mpc * OR_MPC_M / OR_C_MS);
}

/* Plus and cross polarisations at frequency f (zero at or above the ISCO):
 *   h+ = A f^(-7/6) (1 + cos^2 iota)/2 exp(-i Psi),   hx = -i A f^(-7/6) cos(iota) exp(-i Psi). */
void or_polarisations(double f, const double* par, double complex* hp, double complex* hc) {
  if (f >= or_f_isco(par[OR_MC], par[OR_Q])) {
    *hp = 0.0;
    *hc = 0.0;
    return;
  }
  double amp = or_amplitude(par[OR_MC], par[OR_DL]) * pow(f, -7.0 / 6.0);
  double complex e = cexp(-I * or_taylorf2_phase(f, par));
  double ci = cos(par[OR_IOTA]);
  *hp = amp * 0.5 * (1.0 + ci * ci) * e;
  *hc = -I * amp * ci * e;
}

/* ------------------------------------------------------------------------------------ */
/* Detector response.  Source direction n = (cos d cos p, cos d sin p, sin d) with
 * p = RA - GMST; wave-frame axes X, Y rotated by the polarisation angle psi; detector
 * tensor D = (x x^T - y y^T)/2; F+ = X.D.X - Y.D.Y, Fx = X.D.Y + Y.D.X.  The paper names
 * two- and three-detector networks (abstract; Sec. III A) but gives no geometry. */
void or_antenna(const double* xarm, const double* yarm, double ra, double dec, double psi, double gmst, double* fp,
                double* fc) {
  double p = ra - gmst;
  double X[3] = {sin(p) * cos(psi) - sin(psi) * cos(p) * sin(dec), -cos(p) * cos(psi) - sin(psi) * sin(p) * sin(dec),
                 sin(psi) * cos(dec)};
  double Y[3] = {-sin(p) * sin(psi) - cos(psi) * cos(p) * sin(dec), cos(p) * sin(psi) - cos(psi) * sin(p) * sin(dec),
                 cos(psi) * cos(dec)};
  double D[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) D[a][b] = 0.5 * (xarm[a] * xarm[b] - yarm[a] * yarm[b]);
  double xdx = 0, ydy = 0, xdy = 0, ydx = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      xdx += X[a] * D[a][b] * X[b];
      ydy += Y[a] * D[a][b] * Y[b];
      xdy += X[a] * D[a][b] * Y[b];
      ydx += Y[a] * D[a][b] * X[b];
    }
  *fp = xdx - ydy;
  *fc = xdy + ydx;
}

/* Arrival-time offset of detector at vertex r relative to the geocentre: -r.n / c */
double or_time_delay(const double* vertex, double ra, double dec, double gmst) {
  double p = ra - gmst;
  double n[3] = {cos(dec) * cos(p), cos(dec) * sin(p), sin(dec)};
  return -(vertex[0] * n[0] + vertex[1] * n[1] + vertex[2] * n[2]) / OR_C_MS;
}

/* Strain of detector d at frequency f: (F+ h+ + Fx hx) exp(-2 pi i f dt). */
double complex or_detector_strain(const or_event* ev, int d, double f, const double* par) {
  double fp, fc;
  or_antenna(ev->xarm + 3 * d, ev->yarm + 3 * d, par[OR_RA], par[OR_DEC], par[OR_PSI], ev->gmst, &fp, &fc);
  double dt = or_time_delay(ev->vertex + 3 * d, par[OR_RA], par[OR_DEC], ev->gmst);
  double complex hp, hc;
  or_polarisations(f, par, &hp, &hc);
  return (fp * hp + fc * hc) * cexp(-I * OR_TWO_PI * f * dt);
}

/* ------------------------------------------------------------------------------------ */
/* log I0(x) for x >= 0: the power series sum (x^2/4)^k / (k!)^2 below x = 30, the
 * Hankel asymptotic expansion e^x / sqrt(2 pi x) sum_k [(2k-1)!!]^2 / (k! (8x)^k)
 * above.  Used by the analytic phase marginalisation (Sec. III). */
double or_log_i0(double x) {
  x = fabs(x);
  if (x < 30.0) {
    double term = 1.0, sum = 1.0, y = 0.25 * x * x;
    for (int k = 1; k < 500; ++k) {
      term *= y / ((double)k * (double)k);
      sum += term;
      if (term < 1e-17 * sum) break;
    }
    return log(sum);
  }
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    double a = (2.0 * k - 1.0);
    term *= a * a / ((double)k * 8.0 * x);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return x - 0.5 * log(OR_TWO_PI * x) + log(sum);
}

/* ------------------------------------------------------------------------------------ */
/* Noise-weighted inner products of Eq. 1 against the data, the likelihood ratio of
 * Eq. 3 (the constant -(d|d)/2 of Eq. 2 is dropped), and its marginalisations.
 *
 * mode none:            ln L = Re(d|h) - (h|h)/2 at the given phi_c and d_L
 * PHASE:                h at phi_c = 0, ln L = ln I0(|Z|) - H/2  (uniform phi_c prior)
 * PHASE|DISTANCE:       Z1, H1 at d_L = 1 Mpc,
 *                       ln L = ln int p(d) I0(|Z1|/d) exp(-H1/(2 d^2)) dd,
 *                       p(d) = 3 d^2 / (dmax^3 - dmin^3) on [dmin, dmax]
 * TIME:                 ln L = ln[(1/J) sum_j exp(Re z_j - H/2)], z_j the overlap with h
 *                       shifted by tau_j = (j - J/2) dt_shift, i.e. h(f) exp(-2 pi i f tau_j);
 *                       t_c is the centre of the window, phi_c is sampled. */

/* log of the distance-marginalised likelihood by adaptive Simpson quadrature */
typedef struct {
  double z1, h1, dmin, dmax, gshift;
} or_dist_ctx;

static double or_dist_log_integrand(const or_dist_ctx* c, double d) {
  double lp = log(3.0 * d * d / (pow(c->dmax, 3) - pow(c->dmin, 3)));
  return lp + or_log_i0(c->z1 / d) - c->h1 / (2.0 * d * d);
}

static double or_dist_f(const or_dist_ctx* c, double d) { return exp(or_dist_log_integrand(c, d) - c->gshift); }

static double or_simpson_rec(const or_dist_ctx* c, double a, double b, double fa, double fm, double fb, double whole,
                             double tol, int depth) {
  double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = or_dist_f(c, lm), frm = or_dist_f(c, rm);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * tol) return left + right + delta / 15.0;
  return or_simpson_rec(c, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         or_simpson_rec(c, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

double or_distance_marginal(double z1, double h1, double dmin, double dmax) {
  or_dist_ctx c = {z1, h1, dmin, dmax, 0.0};
  /* shift by the largest value on a fine scan so the integrand peaks near one */
  const int n_scan = 8192;
  double gmax = -INFINITY;
  for (int i = 0; i <= n_scan; ++i) {
    double d = dmin + (dmax - dmin) * i / n_scan;
    double g = or_dist_log_integrand(&c, d);
    if (g > gmax) gmax = g;
  }
  c.gshift = gmax;
  /* integrate panel by panel so that a narrow peak is never stepped over */
  const int n_panel = 512;
  double total = 0.0;
  for (int i = 0; i < n_panel; ++i) {
    double a = dmin + (dmax - dmin) * i / n_panel, b = dmin + (dmax - dmin) * (i + 1) / n_panel;
    double fa = or_dist_f(&c, a), fb = or_dist_f(&c, b), fm = or_dist_f(&c, 0.5 * (a + b));
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    total += or_simpson_rec(&c, a, b, fa, fm, fb, whole, 1e-15 * (dmax - dmin), 40);
  }
  return gmax + log(total);
}

static int or_valid(const double* par, uint32_t marg) {
  if (!(par[OR_MC] > 0.0) || !(par[OR_Q] > 0.0)) return 0;
  if (!(fabs(par[OR_CHI1]) < 1.0) || !(fabs(par[OR_CHI2]) < 1.0)) return 0;
  if (!(marg & OR_MARG_DISTANCE) && !(par[OR_DL] > 0.0)) return 0;
  for (int i = 0; i < OR_NPAR; ++i)
    if (!isfinite(par[i])) return 0;
  return 1;
}

double or_loglike(const or_event* ev, const double* par_in) {
  uint32_t marg = ev->marg;
  if (!or_valid(par_in, marg)) return -INFINITY;
  double par[OR_NPAR];
  memcpy(par, par_in, sizeof(par));
  if (marg & OR_MARG_PHASE) par[OR_PHIC] = 0.0;
  if (marg & OR_MARG_DISTANCE) par[OR_DL] = 1.0;

  int J = (marg & OR_MARG_TIME) ? ev->n_tshift : 0;
  double complex* zj = NULL;
  if (J > 0) {
    zj = (double complex*)calloc((size_t)J, sizeof(double complex));
    if (!zj) return NAN;
  }
  double complex dh = 0.0;
  double hh = 0.0;
  for (int d = 0; d < ev->n_det; ++d) {
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = or_freq(ev->f_lo, ev->df, k);
      double complex h = or_detector_strain(ev, d, f, par);
      double S = ev->psd[(int64_t)d * ev->n_bins + k];
      const double* s = ev->strain + 2 * ((int64_t)d * ev->n_bins + k);
      double complex data = s[0] + I * s[1];
      double complex prod = 4.0 * ev->df * conj(data) * h / S;
      dh += prod;
      hh += 4.0 * ev->df * creal(conj(h) * h) / S;
      for (int j = 0; j < J; ++j) {
        double tau = (j - J / 2) * ev->dt_shift;
        zj[j] += prod * cexp(-I * OR_TWO_PI * f * tau);
      }
    }
  }
  double out;
  if (marg == 0) {
    out = creal(dh) - 0.5 * hh;
  } else if (marg == OR_MARG_PHASE) {
    out = or_log_i0(cabs(dh)) - 0.5 * hh;
  } else if (marg == (OR_MARG_PHASE | OR_MARG_DISTANCE)) {
    out = or_distance_marginal(cabs(dh), hh, ev->dmin, ev->dmax);
  } else if (marg == OR_MARG_TIME) {
    double mx = -INFINITY;
    for (int j = 0; j < J; ++j)
      if (creal(zj[j]) > mx) mx = creal(zj[j]);
    double s = 0.0;
    for (int j = 0; j < J; ++j) s += exp(creal(zj[j]) - mx);
    out = mx + log(s / J) - 0.5 * hh;
  } else {
    out = NAN; /* unsupported combination */
  }
  free(zj);
  return out;
}

/* par: n x 11 row-major; out: n.  Samples are independent (OpenMP over samples). */
void or_loglike_batch(const or_event* ev, int64_t n, const double* par, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) out[i] = or_loglike(ev, par + OR_NPAR * i);
}

/* Complex overlap Z = sum_det (d|h)_complex and H = sum_det (h|h) at the given parameters
 * (exposed for the pins and for parity diagnostics). */
void or_overlaps(const or_event* ev, const double* par, double* z_re, double* z_im, double* hh_out) {
  double complex dh = 0.0;
  double hh = 0.0;
  for (int d = 0; d < ev->n_det; ++d)
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = or_freq(ev->f_lo, ev->df, k);
      double complex h = or_detector_strain(ev, d, f, par);
      double S = ev->psd[(int64_t)d * ev->n_bins + k];
      const double* s = ev->strain + 2 * ((int64_t)d * ev->n_bins + k);
      dh += 4.0 * ev->df * conj(s[0] + I * s[1]) * h / S;
      hh += 4.0 * ev->df * creal(conj(h) * h) / S;
    }
  *z_re = creal(dh);
  *z_im = cimag(dh);
  *hh_out = hh;
}

/* ------------------------------------------------------------------------------------ */
/* Synthetic data: d = n + h(theta_true) per detector and bin.  Noise (when add_noise):
 * n_k = sqrt(S_k / (4 df)) (g1 + i g2), g1, g2 from Box-Muller on Philox words with
 * counter (k, det, 1, 0) and key = noise seed, so that Var (n|h) = (h|h). */
void or_make_strain(const or_event* ev, const double* par, uint64_t noise_seed, int add_noise, double* strain_out) {
  uint32_t key[2] = {(uint32_t)noise_seed, (uint32_t)(noise_seed >> 32)};
  for (int d = 0; d < ev->n_det; ++d)
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = or_freq(ev->f_lo, ev->df, k);
      double complex h = or_detector_strain(ev, d, f, par);
      if (add_noise) {
        uint32_t ctr[4] = {(uint32_t)k, (uint32_t)d, 1u, 0u}, w[4];
        or_philox4x32_10(ctr, key, w);
        double g1, g2;
        or_box_muller(w[0], w[1], &g1, &g2);
        double sig = sqrt(ev->psd[(int64_t)d * ev->n_bins + k] / (4.0 * ev->df));
        h += sig * (g1 + I * g2);
      }
      strain_out[2 * ((int64_t)d * ev->n_bins + k)] = creal(h);
      strain_out[2 * ((int64_t)d * ev->n_bins + k) + 1] = cimag(h);
    }
}

/* Optimal network SNR^2 = sum_det (h|h) of the template at par. */
double or_optimal_snr2(const or_event* ev, const double* par) {
  double hh = 0.0;
  for (int d = 0; d < ev->n_det; ++d)
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = or_freq(ev->f_lo, ev->df, k);
      double complex h = or_detector_strain(ev, d, f, par);
      hh += 4.0 * ev->df * creal(conj(h) * h) / ev->psd[(int64_t)d * ev->n_bins + k];
    }
  return hh;
}

/* Fisher matrix Gamma_ij = sum_det (d_i h | d_j h) at par by central differences with
 * the given absolute steps, over the parameter slots ids[0..P-1].  This is the metric of
 * the inner product (Sec. II A); the proposal is a Gaussian in it. */
void or_fisher(const or_event* ev, const double* par, int32_t P, const int32_t* ids, const double* steps,
               double* gamma) {
  int64_t nb = ev->n_bins;
  double complex* dh = (double complex*)malloc(sizeof(double complex) * (size_t)P * (size_t)ev->n_det * (size_t)nb);
  if (!dh) return;
  for (int32_t i = 0; i < P; ++i) {
    double pp[OR_NPAR], pm[OR_NPAR];
    memcpy(pp, par, sizeof(pp));
    memcpy(pm, par, sizeof(pm));
    pp[ids[i]] += steps[i];
    pm[ids[i]] -= steps[i];
    for (int d = 0; d < ev->n_det; ++d)
      for (int64_t k = 0; k < nb; ++k) {
        double f = or_freq(ev->f_lo, ev->df, k);
        dh[((int64_t)i * ev->n_det + d) * nb + k] =
            (or_detector_strain(ev, d, f, pp) - or_detector_strain(ev, d, f, pm)) / (2.0 * steps[i]);
      }
  }
  for (int32_t i = 0; i < P; ++i)
    for (int32_t j = 0; j < P; ++j) {
      double s = 0.0;
      for (int d = 0; d < ev->n_det; ++d)
        for (int64_t k = 0; k < nb; ++k)
          s += 4.0 * ev->df *
               creal(conj(dh[((int64_t)i * ev->n_det + d) * nb + k]) * dh[((int64_t)j * ev->n_det + d) * nb + k]) /
               ev->psd[(int64_t)d * nb + k];
      gamma[i * P + j] = s;
    }
  free(dh);
}

/* ------------------------------------------------------------------------------------ */
/* Prior densities of the sampled slots.  The paper assumes "natural priors" for the
 * extrinsics (Sec. III): uniform RA, cos(dec), uniform psi, sin(iota), d_L^2, uniform
 * t_c and phi_c.  Masses: flat in (Mc, q) on the box, or flat in (m1, m2) restricted to
 * the (Mc, q) box (flag OR_PRIOR_M1M2), normalised over the box. */

static double or_q_integrand(double q) { return pow(1.0 + q, 0.4) * pow(q, -1.2); }

static double or_simpson_q(double a, double b, double fa, double fm, double fb, double whole, double tol, int depth) {
  double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = or_q_integrand(lm), frm = or_q_integrand(rm);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * tol) return left + right + delta / 15.0;
  return or_simpson_q(a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         or_simpson_q(m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

/* integral of |d(m1,m2)/d(Mc,q)| over the box */
double or_mass_prior_volume(double mc_lo, double mc_hi, double q_lo, double q_hi) {
  double fa = or_q_integrand(q_lo), fb = or_q_integrand(q_hi), fm = or_q_integrand(0.5 * (q_lo + q_hi));
  double whole = (q_hi - q_lo) / 6.0 * (fa + 4.0 * fm + fb);
  double qint = or_simpson_q(q_lo, q_hi, fa, fm, fb, whole, 1e-16, 50);
  return 0.5 * (mc_hi * mc_hi - mc_lo * mc_lo) * qint;
}

/* log prior of one sample given its P sampled values (theta_i[p] for slot ids[p]) */
double or_log_prior(int32_t P, const int32_t* ids, const double* lo, const double* hi, uint32_t flags,
                    const double* theta_i) {
  double lp = 0.0, mc = NAN, q = NAN;
  int has_mc = 0, has_q = 0;
  double mc_lo = 0, mc_hi = 0, q_lo = 0, q_hi = 0;
  for (int32_t p = 0; p < P; ++p) {
    double x = theta_i[p];
    int id = ids[p];
    switch (id) {
      case OR_RA:
      case OR_PHIC:
        if (!(x >= 0.0 && x < OR_TWO_PI)) return -INFINITY;
        lp -= log(OR_TWO_PI);
        break;
      case OR_PSI:
        if (!(x >= 0.0 && x < OR_PI)) return -INFINITY;
        lp -= log(OR_PI);
        break;
      case OR_DEC:
        if (!(x >= lo[p] && x <= hi[p])) return -INFINITY;
        lp += log(cos(x) / (sin(hi[p]) - sin(lo[p])));
        break;
      case OR_IOTA:
        if (!(x >= lo[p] && x <= hi[p])) return -INFINITY;
        lp += log(sin(x) / (cos(lo[p]) - cos(hi[p])));
        break;
      case OR_DL:
        if (!(x >= lo[p] && x <= hi[p])) return -INFINITY;
        lp += log(3.0 * x * x / (pow(hi[p], 3) - pow(lo[p], 3)));
        break;
      default: /* MC, Q, CHI1, CHI2, TC: flat on the box */
        if (!(x >= lo[p] && x <= hi[p])) return -INFINITY;
        if (id == OR_MC) { mc = x; has_mc = 1; mc_lo = lo[p]; mc_hi = hi[p]; }
        if (id == OR_Q) { q = x; has_q = 1; q_lo = lo[p]; q_hi = hi[p]; }
        if (!((flags & OR_PRIOR_M1M2) && (id == OR_MC || id == OR_Q))) lp -= log(hi[p] - lo[p]);
        break;
    }
  }
  if ((flags & OR_PRIOR_M1M2) && has_mc && has_q)
    lp += log(or_mass_jacobian(mc, q) / or_mass_prior_volume(mc_lo, mc_hi, q_lo, q_hi));
  return lp;
}

/* Proposal draws (the proposal g of Eq. 5): z ~ N(0, I_P), theta = mu + s L z with L the
 * lower Cholesky factor (row-major) of the proposal covariance.  RA and phi_c wrap into
 * [0, 2 pi), psi into [0, pi).  log g is the unwrapped Gaussian density at z:
 *   log g = -z.z/2 - sum ln L_pp - (P/2) ln(2 pi) - P ln s.
 * theta is SoA: theta[p * n + i].  Sample i uses Philox counter ctr0 + i. */
void or_draw(uint64_t seed, uint64_t ctr0, int64_t n, int32_t P, const int32_t* ids, const double* mean,
             const double* chol, double scale, double* theta, double* logq) {
  double logdet = 0.0;
  for (int32_t p = 0; p < P; ++p) logdet += log(chol[p * P + p]);
  for (int64_t i = 0; i < n; ++i) {
    double z[16];
    or_sample_normals(seed, ctr0 + (uint64_t)i, P, z);
    double zz = 0.0;
    for (int32_t p = 0; p < P; ++p) zz += z[p] * z[p];
    for (int32_t p = 0; p < P; ++p) {
      double x = mean[p];
      for (int32_t r = 0; r <= p; ++r) x += scale * chol[p * P + r] * z[r];
      if (ids[p] == OR_RA || ids[p] == OR_PHIC) {
        x = fmod(x, OR_TWO_PI);
        if (x < 0.0) x += OR_TWO_PI;
        if (x >= OR_TWO_PI) x -= OR_TWO_PI;
      } else if (ids[p] == OR_PSI) {
        x = fmod(x, OR_PI);
        if (x < 0.0) x += OR_PI;
        if (x >= OR_PI) x -= OR_PI;
      }
      theta[(int64_t)p * n + i] = x;
    }
    logq[i] = -0.5 * zz - logdet - 0.5 * P * log(OR_TWO_PI) - P * log(scale);
  }
}

/* Weighted mean and covariance of samples (the refit of the Gaussian proposal from the
 * weighted samples suggested in Sec. III A), two passes.  Periodic slots (RA, phi_c: 2 pi,
 * psi: pi) are taken as offsets from ref wrapped into [-period/2, period/2); the mean is
 * wrapped back into the period.  theta SoA [P][n]; weights <= 0 are skipped. */
void or_weighted_moments(int64_t n, int32_t P, const int32_t* ids, const double* theta, const double* w,
                         const double* ref, double* mean_out, double* cov_out) {
  double period[16], wsum = 0.0, mu[16];
  for (int32_t p = 0; p < P; ++p) {
    period[p] = (ids[p] == OR_PSI) ? OR_PI : (ids[p] == OR_RA || ids[p] == OR_PHIC) ? OR_TWO_PI : 0.0;
    mu[p] = 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!(w[i] > 0.0)) continue;
    wsum += w[i];
    for (int32_t p = 0; p < P; ++p) {
      double d = theta[(int64_t)p * n + i] - ref[p];
      if (period[p] > 0.0) d -= period[p] * floor(d / period[p] + 0.5);
      mu[p] += w[i] * d;
    }
  }
  for (int32_t p = 0; p < P; ++p) mu[p] /= wsum;
  for (int32_t p = 0; p < P; ++p)
    for (int32_t q = 0; q < P; ++q) cov_out[p * P + q] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(w[i] > 0.0)) continue;
    double d[16];
    for (int32_t p = 0; p < P; ++p) {
      double x = theta[(int64_t)p * n + i] - ref[p];
      if (period[p] > 0.0) x -= period[p] * floor(x / period[p] + 0.5);
      d[p] = x - mu[p];
    }
    for (int32_t p = 0; p < P; ++p)
      for (int32_t q = 0; q < P; ++q) cov_out[p * P + q] += w[i] * d[p] * d[q] / wsum;
  }
  for (int32_t p = 0; p < P; ++p) {
    double x = ref[p] + mu[p];
    if (period[p] > 0.0) x -= period[p] * floor(x / period[p]);
    mean_out[p] = x;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Importance weights (Eq. 5), Kish effective sample size (Eq. 6) and the evidence.
 *   log w_i = log L_i + log pi_i - log g_i
 *   m = max log w,  S1 = sum e^(log w - m),  S2 = sum e^(2 (log w - m))
 *   ESS = S1^2 / S2,  log Z = m + ln S1 - ln N  (N counts every draw),
 *   w_i (normalised) = e^(log w_i - m) / S1.
 * Two passes, sums in long double.  out = {ess, log_z, m, n, s1, s2}. */
void or_reduce(int64_t n, const double* loglike, const double* logp, const double* logq, double* w_out, double* out) {
  double m = -INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double lw = loglike[i] + logp[i] - logq[i];
    if (lw > m) m = lw;
  }
  long double s1 = 0.0L, s2 = 0.0L;
  if (m > -INFINITY) {
    for (int64_t i = 0; i < n; ++i) {
      double lw = loglike[i] + logp[i] - logq[i];
      long double e = expl((long double)lw - (long double)m);
      s1 += e;
      s2 += e * e;
    }
  }
  if (w_out)
    for (int64_t i = 0; i < n; ++i) {
      double lw = loglike[i] + logp[i] - logq[i];
      w_out[i] = (m > -INFINITY) ? (double)(expl((long double)lw - (long double)m) / s1) : 0.0;
    }
  out[0] = (s2 > 0.0L) ? (double)(s1 * s1 / s2) : 0.0;
  out[1] = (m > -INFINITY) ? m + (double)logl((long double)s1) - log((double)n) : -INFINITY;
  out[2] = m;
  out[3] = (double)n;
  out[4] = (double)s1;
  out[5] = (double)s2;
}

/* ------------------------------------------------------------------------------------ */
/* Tiled proposal (Sec. II; App. A): a template bank spans the space of waveforms, every
 * prior sample belongs to the tile of the template it matches best, and the proposal
 * draws a tile with probability proportional to its share of the prior volume times the
 * likelihood at its template, then a prior sample of that tile.
 *
 * The space is the two-parameter demonstration of App. A: a sampled chirp-mass coordinate
 * x, mapped to the chirp mass mc_base + mod(x, mc_period) (the "cyclic chirp mass"; a
 * period <= 0 keeps Mc = x), and a sampled mass ratio q that may fall below one, q and 1/q
 * naming the same binary; spins are fixed.  Readings where the paper is silent: the match
 * is the normalised overlap maximised over phase at a common coalescence time (the 2-D
 * likelihood it tiles samples neither time nor phase); the noise weighting is one PSD; a
 * waveform is zero at and above its ISCO as in the likelihood. */
typedef struct {
  double x_lo, x_hi;
  double mc_period, mc_base;
  double q_lo, q_hi;
  double chi1, chi2;
  double f_lo, df;
  int32_t n_bins;
  const double* psd; /* [n_bins] */
} or_tiling;

/* Physical chirp mass and mass ratio (>= 1) of a point of the sampled space. */
void or_tiling_physical(const or_tiling* t, double x, double q, double* mc, double* qp) {
  if (t->mc_period > 0.0) {
    double r = fmod(x, t->mc_period);
    if (r < 0.0) r += t->mc_period;
    *mc = t->mc_base + r;
  } else {
    *mc = x;
  }
  *qp = (q >= 1.0) ? q : 1.0 / q;
}

/* Whitened, unit-norm waveform of one point: u_k = f_k^(-7/6) e^(-i Psi(f_k)) / sqrt(S_k),
 * divided by sqrt(sum_k |.|^2), zero at and above the ISCO.  Returns the number of live
 * bins (0: no bin below the ISCO, u is all zero). */
int32_t or_tiling_waveform(const or_tiling* t, double x, double q, double complex* u) {
  double par[OR_NPAR];
  memset(par, 0, sizeof par);
  or_tiling_physical(t, x, q, &par[OR_MC], &par[OR_Q]);
  par[OR_CHI1] = t->chi1;
  par[OR_CHI2] = t->chi2;
  par[OR_DL] = 1.0;
  double fi = or_f_isco(par[OR_MC], par[OR_Q]), norm2 = 0.0;
  int32_t live = 0;
  for (int32_t k = 0; k < t->n_bins; ++k) {
    double f = or_freq(t->f_lo, t->df, k);
    if (f >= fi) {
      u[k] = 0.0;
      continue;
    }
    double a = pow(f, -7.0 / 6.0) / sqrt(t->psd[k]);
    u[k] = a * cexp(-I * or_taylorf2_phase(f, par));
    norm2 += a * a;
    ++live;
  }
  if (live == 0) return 0;
  double inv = 1.0 / sqrt(norm2);
  for (int32_t k = 0; k < t->n_bins; ++k) u[k] *= inv;
  return live;
}

/* |sum_k conj(u_a,k) u_b,k| of two unit-norm waveforms: the overlap (a|b) / sqrt((a|a)(b|b))
 * of Eq. 1's inner product maximised over a constant phase (the maximum over phi of
 * Re(e^(i phi) z) is |z|). */
double or_tiling_overlap(int32_t n_bins, const double complex* ua, const double complex* ub) {
  double complex z = 0.0;
  for (int32_t k = 0; k < n_bins; ++k) z += conj(ua[k]) * ub[k];
  return cabs(z);
}

double or_tiling_match(const or_tiling* t, double xa, double qa, double xb, double qb) {
  double complex* ua = (double complex*)malloc(sizeof(double complex) * (size_t)t->n_bins);
  double complex* ub = (double complex*)malloc(sizeof(double complex) * (size_t)t->n_bins);
  double m = 0.0;
  if (or_tiling_waveform(t, xa, qa, ua) > 0 && or_tiling_waveform(t, xb, qb, ub) > 0)
    m = or_tiling_overlap(t->n_bins, ua, ub);
  free(ua);
  free(ub);
  return m;
}

/* Stochastic template placement (App. A "Template bank generation"; the stochastic
 * method the paper adopts): candidates are visited in the given order; one joins the bank
 * when its match with every template already in the bank is below min_match.  Placement
 * stops after stop_after consecutive rejections, at max_templates, or when the candidates
 * run out.  Candidates without a live bin are skipped (counted as rejections).
 * cand is [2][n_cand] (x row, q row).  Writes the indices of the accepted candidates to
 * idx_out, the number of candidates visited to *n_used and, when margin is non-null, the
 * smallest |match - min_match| of any decision taken.  Returns the bank size. */
int32_t or_tiling_bank(const or_tiling* t, int64_t n_cand, const double* cand, double min_match, int64_t stop_after,
                       int32_t max_templates, int32_t* idx_out, int64_t* n_used, double* margin) {
  const size_t nb = (size_t)t->n_bins;
  double complex* bank =
      (double complex*)malloc(sizeof(double complex) * nb * (size_t)(max_templates > 0 ? max_templates : 1));
  double complex* u = (double complex*)malloc(sizeof(double complex) * nb);
  int32_t T = 0;
  int64_t run = 0, i = 0;
  double mg = INFINITY;
  for (; i < n_cand && T < max_templates && run < stop_after; ++i) {
    if (or_tiling_waveform(t, cand[i], cand[n_cand + i], u) == 0) {
      ++run;
      continue;
    }
    double best = 0.0;
    for (int32_t j = 0; j < T; ++j) {
      double m = or_tiling_overlap(t->n_bins, bank + (size_t)j * nb, u);
      if (m > best) best = m;
    }
    if (T > 0 && fabs(best - min_match) < mg) mg = fabs(best - min_match);
    if (T == 0 || best < min_match) {
      memcpy(bank + (size_t)T * nb, u, sizeof(double complex) * nb);
      idx_out[T++] = (int32_t)i;
      run = 0;
    } else {
      ++run;
    }
  }
  *n_used = i;
  if (margin) *margin = mg;
  free(bank);
  free(u);
  return T;
}

/* Tile of each point (App. A "Tiling the prior volume"): the template of highest match,
 * the lowest index among equal matches; -1 for a point without a live bin.  pts is [2][n],
 * tpl is [2][T].  match_out gets the best match, second_out (nullable) the runner-up. */
void or_tiling_assign(const or_tiling* t, int64_t n, const double* pts, int32_t T, const double* tpl,
                      int32_t* tile_out, double* match_out, double* second_out) {
  const size_t nb = (size_t)t->n_bins;
  double complex* tw = (double complex*)malloc(sizeof(double complex) * nb * (size_t)(T > 0 ? T : 1));
  int32_t* tlive = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
  for (int32_t j = 0; j < T; ++j) tlive[j] = or_tiling_waveform(t, tpl[j], tpl[T + j], tw + (size_t)j * nb);
#pragma omp parallel
  {
    double complex* u = (double complex*)malloc(sizeof(double complex) * nb);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int32_t best_j = -1;
      double best = -1.0, second = -1.0;
      if (or_tiling_waveform(t, pts[i], pts[n + i], u) > 0) {
        for (int32_t j = 0; j < T; ++j) {
          double m = tlive[j] > 0 ? or_tiling_overlap(t->n_bins, tw + (size_t)j * nb, u) : 0.0;
          if (m > best) {
            second = best;
            best = m;
            best_j = j;
          } else if (m > second) {
            second = m;
          }
        }
      }
      tile_out[i] = best_j;
      match_out[i] = best_j >= 0 ? best : 0.0;
      if (second_out) second_out[i] = second > 0.0 ? second : 0.0;
    }
    free(u);
  }
  free(tw);
  free(tlive);
}

/* Tiles as lists: count of each tile, exclusive offsets and the members of every tile in
 * increasing sample order.  tile has n entries in [-1, T); -1 belongs to no tile. */
void or_tiling_lists(int64_t n, const int32_t* tile, int32_t T, int64_t* count, int64_t* offset, int64_t* members) {
  for (int32_t j = 0; j < T; ++j) count[j] = 0;
  for (int64_t i = 0; i < n; ++i)
    if (tile[i] >= 0) ++count[tile[i]];
  int64_t o = 0;
  for (int32_t j = 0; j < T; ++j) {
    offset[j] = o;
    o += count[j];
  }
  int64_t* fill = (int64_t*)calloc((size_t)(T > 0 ? T : 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    if (tile[i] >= 0) members[offset[tile[i]] + fill[tile[i]]++] = i;
  free(fill);
}

/* Mixture over tiles (Sec. II; App. A "Generation of the posterior distribution"): tile j
 * is drawn with probability p_j proportional to (n_j / N) L_j, its share of the prior
 * volume (n_j of the N prior samples) times the likelihood ratio at its template.  Kept
 * unnormalised and shifted: c_j = sum_{i <= j} n_i exp(lnL_i - m), m = max over tiles with
 * n_i > 0 of lnL_i.  Returns m; c has T entries (the last one is the total). */
double or_tiling_mixture(int32_t T, const int64_t* count, const double* loglike_tpl, double* c) {
  double m = -INFINITY;
  for (int32_t j = 0; j < T; ++j)
    if (count[j] > 0 && loglike_tpl[j] > m) m = loglike_tpl[j];
  double s = 0.0;
  for (int32_t j = 0; j < T; ++j) {
    if (count[j] > 0) s += (double)count[j] * exp(loglike_tpl[j] - m);
    c[j] = s;
  }
  return m;
}

/* Draws from the mixture.  Draw i takes the Philox4x32-10 block of counter
 * (lo g, hi g, 3, 0), g = ctr0 + i, under the key (seed lo, seed hi).  Words (r0, r1) give
 * u = ((r0 2^32 + r1) >> 11) 2^-53 in [0, 1), and the tile is the first j with
 * c_j > u c_(T-1).  Words (r2, r3) give a 64-bit integer r, and the member is the
 * ((r n_j) >> 64)-th of the tile's list (multiply-shift: uniform up to n_j / 2^64).  For
 * the drawn prior sample,
 *   ln g = ln pi + ln p_j - ln(n_j / N) = ln pi + lnL_j - m - ln c_(T-1) + ln N,
 * the proposal density being the prior density scaled by p_j / (n_j / N) inside tile j.
 * Writes the pool index and tile of every draw and ln g - ln pi. */
void or_tiling_draw(uint64_t seed, uint64_t ctr0, int64_t n, int32_t T, const double* c, double m,
                    const double* loglike_tpl, const int64_t* count, const int64_t* offset, const int64_t* members,
                    int64_t n_pool, int64_t* pool_idx, int32_t* tile_out, double* log_ratio) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double total = c[T - 1];
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t g = ctr0 + (uint64_t)i;
    const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), 3u, 0u};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    const uint64_t w0 = ((uint64_t)r[0] << 32) | r[1];
    const double u = (double)(w0 >> 11) * (1.0 / 9007199254740992.0);
    const double target = u * total;
    int32_t j = 0;
    while (j < T - 1 && !(c[j] > target)) ++j;
    const uint64_t w1 = ((uint64_t)r[2] << 32) | r[3];
    const uint64_t k = (uint64_t)(((unsigned __int128)w1 * (unsigned __int128)(uint64_t)count[j]) >> 64);
    pool_idx[i] = members[offset[j] + (int64_t)k];
    tile_out[i] = j;
    log_ratio[i] = loglike_tpl[j] - m - log(total) + log((double)n_pool);
  }
}

/* ------------------------------------------------------------------------------------ */
/* Credible level of a reference point (the P-P self-consistency test of Sec. III A): for
 * every sampled slot p, the weighted fraction of the posterior below the reference,
 *   level_p = [sum_i w_i 1(theta_pi < ref_p) + 1/2 sum_i w_i 1(theta_pi = ref_p)] / sum_i w_i,
 * with the importance weights w_i (Eq. 5; any positive scale).  Over sources drawn from the
 * prior and analysed with the same prior, the level of the true value is uniform on [0, 1].
 * theta is SoA [P][n]; sums in long double. */
void or_credible_levels(int64_t n, int32_t P, const double* theta, const double* w, const double* ref, double* out) {
  long double tot = 0.0L;
  for (int64_t i = 0; i < n; ++i)
    if (w[i] > 0.0) tot += w[i];
  for (int32_t p = 0; p < P; ++p) {
    long double below = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
      if (!(w[i] > 0.0)) continue;
      const double x = theta[(int64_t)p * n + i];
      if (x < ref[p])
        below += w[i];
      else if (x == ref[p])
        below += 0.5L * w[i];
    }
    out[p] = tot > 0.0L ? (double)(below / tot) : NAN;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Relative binning (the heterodyned likelihood of Zackay, Dai & Venumadhav 2018, one of the
 * faster likelihoods the paper notes its method can use, Sec. IV): near a fiducial par0 the
 * ratio r(f) = h(f; par) / h(f; par0) of detector strains (without the ISCO cut) is smooth,
 * so within each coarse bin [f_b, f_b+1) it is replaced by its chord through the bin's two
 * edges:  (d|h) ~ sum_det sum_b sum_{k in b, f_k < f_isco} 4 df conj(d_k) h0_k / S_k
 *                 * [r(f_b) + (f_k - f_b) (r(f_b+1) - r(f_b)) / (f_b+1 - f_b)].
 * (h|h) is kept exact (the amplitude is analytic).  edges: n_rb + 1 increasing bin indices,
 * edges[0] = 0, edges[n_rb] = n_bins (the last edge is the frequency one past the grid).
 * Marginalisation as or_loglike (time marginalisation is not supported: NaN). */
static double complex or_detector_strain_uncut(const or_event* ev, int d, double f, const double* par) {
  double fp, fc;
  or_antenna(ev->xarm + 3 * d, ev->yarm + 3 * d, par[OR_RA], par[OR_DEC], par[OR_PSI], ev->gmst, &fp, &fc);
  double dt = or_time_delay(ev->vertex + 3 * d, par[OR_RA], par[OR_DEC], ev->gmst);
  double amp = or_amplitude(par[OR_MC], par[OR_DL]) * pow(f, -7.0 / 6.0);
  double complex e = cexp(-I * or_taylorf2_phase(f, par));
  double ci = cos(par[OR_IOTA]);
  double complex hp = amp * 0.5 * (1.0 + ci * ci) * e, hc = -I * amp * ci * e;
  return (fp * hp + fc * hc) * cexp(-I * OR_TWO_PI * f * dt);
}

double or_rb_loglike(const or_event* ev, const double* par0_in, int32_t n_rb, const int32_t* edges,
                     const double* par_in) {
  uint32_t marg = ev->marg;
  if ((marg & OR_MARG_TIME) || n_rb < 1) return NAN;
  if (!or_valid(par_in, marg)) return -INFINITY;
  double par[OR_NPAR], par0[OR_NPAR];
  memcpy(par, par_in, sizeof(par));
  memcpy(par0, par0_in, sizeof(par0));
  if (marg & OR_MARG_PHASE) par[OR_PHIC] = par0[OR_PHIC] = 0.0;
  if (marg & OR_MARG_DISTANCE) par[OR_DL] = par0[OR_DL] = 1.0;
  const double fi = or_f_isco(par[OR_MC], par[OR_Q]);
  double complex dh = 0.0;
  double hh = 0.0;
  for (int d = 0; d < ev->n_det; ++d) {
    for (int32_t b = 0; b < n_rb; ++b) {
      const int64_t k0 = edges[b], k1 = edges[b + 1];
      const double fb = or_freq(ev->f_lo, ev->df, k0), fb1 = or_freq(ev->f_lo, ev->df, k1);
      const double complex h0b = or_detector_strain_uncut(ev, d, fb, par0);
      const double complex h0b1 = or_detector_strain_uncut(ev, d, fb1, par0);
      if (cabs(h0b) == 0.0 || cabs(h0b1) == 0.0) continue; /* a detector blind to the source */
      const double complex rb = or_detector_strain_uncut(ev, d, fb, par) / h0b;
      const double complex rb1 = or_detector_strain_uncut(ev, d, fb1, par) / h0b1;
      const double complex slope = (rb1 - rb) / (fb1 - fb);
      for (int64_t k = k0; k < k1; ++k) {
        const double f = or_freq(ev->f_lo, ev->df, k);
        if (f >= fi) continue;
        const double S = ev->psd[(int64_t)d * ev->n_bins + k];
        const double* s = ev->strain + 2 * ((int64_t)d * ev->n_bins + k);
        const double complex h0 = or_detector_strain_uncut(ev, d, f, par0);
        dh += 4.0 * ev->df * conj(s[0] + I * s[1]) * h0 * (rb + (f - fb) * slope) / S;
      }
    }
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      const double f = or_freq(ev->f_lo, ev->df, k);
      const double complex h = or_detector_strain(ev, d, f, par);
      hh += 4.0 * ev->df * creal(conj(h) * h) / ev->psd[(int64_t)d * ev->n_bins + k];
    }
  }
  if (marg == 0) return creal(dh) - 0.5 * hh;
  if (marg == OR_MARG_PHASE) return or_log_i0(cabs(dh)) - 0.5 * hh;
  if (marg == (OR_MARG_PHASE | OR_MARG_DISTANCE)) return or_distance_marginal(cabs(dh), hh, ev->dmin, ev->dmax);
  return NAN;
}

void or_rb_loglike_batch(const or_event* ev, const double* par0, int32_t n_rb, const int32_t* edges, int64_t n,
                         const double* par, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) out[i] = or_rb_loglike(ev, par0, n_rb, edges, par + OR_NPAR * i);
}
