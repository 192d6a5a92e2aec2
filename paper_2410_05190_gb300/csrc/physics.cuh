// physics.cuh -- FP64 source-model and detector-response formulas of the CUDA path
// (host and device).  The paper models signals with IMRPhenom families (Sec. III); this
// implementation uses the closed-form TaylorF2 aligned-spin inspiral:
//   h+(f) = A f^(-7/6) (1 + cos^2 i)/2 e^(-i Psi(f)),  hx(f) = -i A f^(-7/6) cos i e^(-i Psi(f)),
//   Psi(f) = 2 pi f t_c - phi_c - pi/4 + 3/(128 eta v^5) sum_n phi_n v^n,  v = (pi M f)^(1/3),
// zero at and above the Schwarzschild ISCO of the total mass.  Coefficients: Buonanno et
// al. (2009) non-spinning, Khan et al. (2016, App. B) chi_s / chi_a spin terms; the
// 2.5PN log term is (1 + 3 ln v); spin-cubed and kappa != 1 terms are omitted.
//
// The phase is written as a linear combination of nine fixed functions of frequency,
//   Psi(f) / (2 pi) = c + sum_j C_j B_j(f),
//   B = { f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f, f^2/3, f },
// so that per-event tables of B_j and per-sample coefficients C_j carry all of it.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define MBIS_HD __host__ __device__ __forceinline__
#else
#define MBIS_HD inline
#endif

namespace mbis {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kTsun = 4.925490947641267e-6;             // G Msun / c^3, s (IAU 2015)
constexpr double kClight = 299792458.0;                    // m / s
constexpr double kInvClight = 1.0 / kClight;               // a product, not an FP64 division, per delay
constexpr double kMpcSeconds = 3.0856775814913673e22 / 299792458.0;  // 1 Mpc / c, s
constexpr double kEulerGamma = 0.577215664901532860606512090082;
constexpr int kNumBasis = 9;
constexpr int kNumSlots = 11;

enum Slot { kMc = 0, kQ, kChi1, kChi2, kRa, kDec, kPsi, kIota, kDl, kTc, kPhic };

// Phase of the model in turns: Psi(f)/(2 pi) = cst + sum_j C[j] * basis_j(f).
struct PhaseCoeffs {
  double C[kNumBasis];
  double cst;
};

MBIS_HD double total_mass_seconds(double mc, double q) {
  // M = Mc (1+q)^(6/5) q^(-3/5)
  return mc * kTsun * pow(1.0 + q, 1.2) * pow(q, -0.6);
}

// The PN phase coefficients' mass-ratio and spin factors (eta, delta = (m1 - m2) / M, chi_s,
// chi_a): phi2, phi3, phi4, the 2.5PN factor c5 (phi5(v) = c5 (1 + 3 ln v)), the 3PN constant
// a6 (phi6(v) = a6 - (6848/21) ln v) and phi7.
struct PNTerms {
  double phi2, phi3, phi4, c5, a6, phi7;
};

MBIS_HD PNTerms pn_terms(double eta, double dm, double xs, double xa) {
  const double e2 = eta * eta, e3 = e2 * eta, pi2 = kPi * kPi;
  constexpr double kLn4 = 1.3862943611198906188344642429164;
  PNTerms t;
  t.phi2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
  t.phi3 = -16.0 * kPi + 113.0 / 3.0 * dm * xa + (113.0 / 3.0 - 76.0 / 3.0 * eta) * xs;
  t.phi4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * e2 +
           (-405.0 / 8.0 + 200.0 * eta) * xa * xa - 405.0 / 4.0 * dm * xa * xs +
           (-405.0 / 8.0 + 5.0 / 2.0 * eta) * xs * xs;
  t.c5 = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) + dm * (-732985.0 / 2268.0 - 140.0 / 9.0 * eta) * xa +
         (-732985.0 / 2268.0 + 24260.0 / 81.0 * eta + 340.0 / 9.0 * e2) * xs;
  t.a6 = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 - 6848.0 / 21.0 * (kEulerGamma + kLn4) +
         (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) * eta + 76055.0 / 1728.0 * e2 - 127825.0 / 1296.0 * e3 +
         kPi * (2270.0 / 3.0 * dm * xa + (2270.0 / 3.0 - 520.0 * eta) * xs) +
         (75515.0 / 144.0 - 8225.0 / 18.0 * eta) * dm * xa * xs +
         (75515.0 / 288.0 - 263245.0 / 252.0 * eta - 480.0 * e2) * xa * xa +
         (75515.0 / 288.0 - 232415.0 / 504.0 * eta + 1255.0 / 9.0 * e2) * xs * xs;
  t.phi7 = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * e2) +
           (-25150083775.0 / 3048192.0 + 10566655595.0 / 762048.0 * eta - 1042165.0 / 3024.0 * e2 +
            5345.0 / 36.0 * e3) * xs +
           dm * (-25150083775.0 / 3048192.0 + 26804935.0 / 6048.0 * eta - 1985.0 / 48.0 * e2) * xa;
  return t;
}

// a = pi M (M the total mass in seconds), la = ln a, a13 = a^(1/3), taken by the caller
MBIS_HD PhaseCoeffs phase_coeffs_a(double q, double chi1, double chi2, double tc, double phic, double a, double la,
                                   double a13) {
  const double eta = q / ((1.0 + q) * (1.0 + q));
  const double dm = (q - 1.0) / (q + 1.0);  // (m1 - m2) / M
  const PNTerms t = pn_terms(eta, dm, 0.5 * (chi1 + chi2), 0.5 * (chi1 - chi2));

  // v = (a f)^(1/3) with a = pi M;  v^n = a^(n/3) f^(n/3);  3 ln v = ln a + ln f
  const double a23 = a13 * a13;
  const double pre = 3.0 / (128.0 * eta) / kTwoPi;  // turns
  PhaseCoeffs pc;
  pc.C[0] = pre / (a23 * a23 * a13);                 // a^(-5/3)   f^(-5/3)
  pc.C[1] = pre * t.phi2 / a;                        // a^(-1)     f^(-1)
  pc.C[2] = pre * t.phi3 / a23;                      // a^(-2/3)   f^(-2/3)
  pc.C[3] = pre * t.phi4 / a13;                      // a^(-1/3)   f^(-1/3)
  pc.C[4] = pre * t.c5;                              // ln f
  pc.C[5] = pre * a13 * (t.a6 - 6848.0 / 63.0 * la); // f^(1/3)
  pc.C[6] = -pre * a13 * (6848.0 / 63.0);            // f^(1/3) ln f
  pc.C[7] = pre * t.phi7 * a23;                      // f^(2/3)
  pc.C[8] = tc;                                      // f
  pc.cst = -phic / kTwoPi - 0.125 + pre * t.c5 * (1.0 + la);
  return pc;
}

// m_sec: total mass in seconds, total_mass_seconds(mc, q)
MBIS_HD PhaseCoeffs phase_coeffs_m(double mc, double q, double chi1, double chi2, double tc, double phic,
                                   double m_sec) {
  (void)mc;
  const double a = kPi * m_sec;
  return phase_coeffs_a(q, chi1, chi2, tc, phic, a, log(a), cbrt(a));
}

MBIS_HD PhaseCoeffs phase_coeffs(double mc, double q, double chi1, double chi2, double tc, double phic) {
  return phase_coeffs_m(mc, q, chi1, chi2, tc, phic, total_mass_seconds(mc, q));
}

MBIS_HD double basis(int j, double f) {
  const double c = cbrt(f);
  switch (j) {
    case 0: return 1.0 / (f * c * c);
    case 1: return 1.0 / f;
    case 2: return 1.0 / (c * c);
    case 3: return 1.0 / c;
    case 4: return log(f);
    case 5: return c;
    case 6: return c * log(f);
    case 7: return c * c;
    default: return f;
  }
}

// all nine basis functions at f, each bit-identical to basis(j, f)
MBIS_HD void basis_all(double f, double* b) {
  const double c = cbrt(f), lf = log(f);
  b[0] = 1.0 / (f * c * c);
  b[1] = 1.0 / f;
  b[2] = 1.0 / (c * c);
  b[3] = 1.0 / c;
  b[4] = lf;
  b[5] = c;
  b[6] = c * lf;
  b[7] = c * c;
  b[8] = f;
}

// d basis_j / df
MBIS_HD double basis_deriv(int j, double f) {
  const double c = cbrt(f);
  switch (j) {
    case 0: return -5.0 / 3.0 / (f * f * c * c);
    case 1: return -1.0 / (f * f);
    case 2: return -2.0 / 3.0 / (f * c * c);
    case 3: return -1.0 / 3.0 / (f * c);
    case 4: return 1.0 / f;
    case 5: return 1.0 / (3.0 * c * c);
    case 6: return (log(f) / 3.0 + 1.0) / (c * c);
    case 7: return 2.0 / 3.0 / c;
    default: return 1.0;
  }
}

// 1 / (6^(3/2) pi M), M in seconds
MBIS_HD double f_isco_m(double m_sec) { return 1.0 / (14.696938456699067 * kPi * m_sec); }

MBIS_HD double f_isco(double mc, double q) { return f_isco_m(total_mass_seconds(mc, q)); }

// number of grid points f_lo + k df (k < n_bins) strictly below the ISCO of total mass m_sec
MBIS_HD int32_t live_bins_m(double m_sec, double f_lo, double df, int32_t n_bins) {
  const double fi = f_isco_m(m_sec);
  double kk = ceil((fi - f_lo) / df);
  if (!(kk > 0.0)) return 0;
  if (kk > (double)n_bins) kk = (double)n_bins;
  int32_t k = (int32_t)kk;
  while (k > 0 && f_lo + (double)(k - 1) * df >= fi) --k;
  while (k < n_bins && f_lo + (double)k * df < fi) ++k;
  return k;
}

MBIS_HD int32_t live_bins(double mc, double q, double f_lo, double df, int32_t n_bins) {
  return live_bins_m(total_mass_seconds(mc, q), f_lo, df, n_bins);
}

// A = sqrt(5/24) pi^(-2/3) (Mc T_sun)^(5/6) / (d_L / c)
MBIS_HD double amplitude(double mc, double dl_mpc) {
  return 0.45643546458763845 * 0.46619407703541166 * pow(mc * kTsun, 5.0 / 6.0) / (dl_mpc * kMpcSeconds);
}

// Antenna patterns of an interferometer with unit arms x, y for a source at (ra, dec)
// with polarisation angle psi:  F+ = ((x.X)^2 - (x.Y)^2 - (y.X)^2 + (y.Y)^2) / 2,
// Fx = (x.X)(x.Y) - (y.X)(y.Y), the contraction of D = (x x - y y)/2 with the wave
// tensors X X - Y Y and X Y + Y X.
MBIS_HD void antenna(const double* x, const double* y, double ra, double dec, double psi, double gmst,
                     double* fp, double* fc) {
  double sp, cp, sd, cd, ss, cs;
  const double ph = ra - gmst;
  sp = sin(ph); cp = cos(ph); sd = sin(dec); cd = cos(dec); ss = sin(psi); cs = cos(psi);
  const double X0 = sp * cs - ss * cp * sd, X1 = -cp * cs - ss * sp * sd, X2 = ss * cd;
  const double Y0 = -sp * ss - cs * cp * sd, Y1 = cp * ss - cs * sp * sd, Y2 = cs * cd;
  const double xX = x[0] * X0 + x[1] * X1 + x[2] * X2, xY = x[0] * Y0 + x[1] * Y1 + x[2] * Y2;
  const double yX = y[0] * X0 + y[1] * X1 + y[2] * X2, yY = y[0] * Y0 + y[1] * Y1 + y[2] * Y2;
  *fp = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
  *fc = xX * xY - yX * yY;
}

// 1/x to FP64 accuracy from an FP32 reciprocal refined by two Newton steps (four FMA; x and
// 1/x inside the FP32 range).  A library FP64 division costs about twice as much, and the
// GB300 runs FP64 at ~1/64 of FP32.
MBIS_HD float rcp_f32(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}

MBIS_HD double rcp_refined(double x) {
  double r = (double)rcp_f32((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// Per-sample set-up of the mixed-precision likelihood kernels: amplitude, phase coefficients
// (the same series as phase_coeffs_a, to FP64 rounding) and ISCO cut, with four reciprocals
// and one FP64 logarithm.  A power or root is seeded in FP32 and refined by one Newton step
// written as a correction, y -= (y^n - x) / (n y^(n-1)), whose small numerator makes an FP32
// divisor enough: the seed's ~1e-7 relative error squares.
//   M = Mc T_sun u^(3/5), u = (1 + q)^2 / q = q + 2 + 1/q = 1/eta:  y = u^(3/5) solves y^5 = u^3
//   a = pi M, a^(1/3) solves y^3 = a;  a^(-n/3) from 1/a and a^(1/3)
//   A = K (Mc T_sun)^(5/6) / d_L:  z = x^(5/6) solves z^6 = x^5
//   f_isco = 1 / (6^(3/2) a)
// (log L of a poor sample can reach 10^4 in magnitude, so A and H keep ~1e-14 accuracy.)
struct SampleSetup {
  PhaseCoeffs pc;
  double amp;    // A at d_L = dl_mpc
  int32_t kcut;  // grid points f_lo + k df strictly below the ISCO
};

MBIS_HD SampleSetup sample_setup(double mc, double q, double chi1, double chi2, double tc, double phic,
                                 double dl_mpc, double f_lo, double df, int32_t n_bins) {
  SampleSetup o;
  const double w = rcp_refined(1.0 + q);
  const double u = q + 2.0 + rcp_refined(q), u3 = u * u * u;
  const double eta = q * w * w, dm = (q - 1.0) * w;
  double y = (double)powf((float)u, 0.6f);
  {
    const double y2 = y * y, y4 = y2 * y2;
    y -= (y4 * y - u3) * (0.2 * (double)rcp_f32((float)y4));
  }
  const double a = kPi * kTsun * mc * y;
  const double la = log(a);
  double a13 = (double)cbrtf((float)a);
  {
    const double c2 = a13 * a13;
    a13 -= (c2 * a13 - a) * ((1.0 / 3.0) * (double)rcp_f32((float)c2));
  }
  const double a23 = a13 * a13, inv_a = rcp_refined(a);
  const double x = mc * kTsun, x2 = x * x, x5 = x2 * x2 * x;
  double z = (double)powf((float)x, 5.0f / 6.0f);
  {
    const double z2 = z * z, z5 = z2 * z2 * z;
    z -= (z5 * z - x5) * ((1.0 / 6.0) * (double)rcp_f32((float)z5));
  }
  o.amp = 0.45643546458763845 * 0.46619407703541166 * z * rcp_refined(dl_mpc * kMpcSeconds);

  const PNTerms t = pn_terms(eta, dm, 0.5 * (chi1 + chi2), 0.5 * (chi1 - chi2));
  const double pre = (3.0 / (256.0 * kPi)) * u;  // 3 / (128 eta) / (2 pi), turns
  const double pa = pre * inv_a;
  o.pc.C[0] = pa * inv_a * a13;                       // a^(-5/3)
  o.pc.C[1] = pa * t.phi2;                            // a^(-1)
  o.pc.C[2] = pa * t.phi3 * a13;                      // a^(-2/3)
  o.pc.C[3] = pa * t.phi4 * a23;                      // a^(-1/3)
  o.pc.C[4] = pre * t.c5;                             // ln f
  o.pc.C[5] = pre * a13 * (t.a6 - 6848.0 / 63.0 * la);
  o.pc.C[6] = -pre * a13 * (6848.0 / 63.0);
  o.pc.C[7] = pre * t.phi7 * a23;
  o.pc.C[8] = tc;
  o.pc.cst = phic * (-1.0 / kTwoPi) - 0.125 + pre * t.c5 * (1.0 + la);

  // the cut: an FP32 estimate of ceil((f_isco - f_lo) / df), then exact FP64 steps to the
  // first grid point at or above f_isco
  const double fi = inv_a * (1.0 / 14.696938456699067);
  const float kf = ceilf((float)(fi - f_lo) * rcp_f32((float)df));
  int32_t k = !(kf > 0.0f) ? 0 : (kf >= (float)n_bins ? n_bins : (int32_t)kf);
  while (k > 0 && f_lo + (double)(k - 1) * df >= fi) --k;
  while (k < n_bins && f_lo + (double)k * df < fi) ++k;
  o.kcut = k;
  return o;
}

// The same two quantities from the sines and cosines of (ra - gmst), dec and psi, so that a
// network evaluates them once per sample.
MBIS_HD void antenna_trig(const double* x, const double* y, double sp, double cp, double sd, double cd, double ss,
                          double cs, double* fp, double* fc) {
  const double X0 = sp * cs - ss * cp * sd, X1 = -cp * cs - ss * sp * sd, X2 = ss * cd;
  const double Y0 = -sp * ss - cs * cp * sd, Y1 = cp * ss - cs * sp * sd, Y2 = cs * cd;
  const double xX = x[0] * X0 + x[1] * X1 + x[2] * X2, xY = x[0] * Y0 + x[1] * Y1 + x[2] * Y2;
  const double yX = y[0] * X0 + y[1] * X1 + y[2] * X2, yY = y[0] * Y0 + y[1] * Y1 + y[2] * Y2;
  *fp = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
  *fc = xX * xY - yX * yY;
}

MBIS_HD double delay_trig(const double* r, double sp, double cp, double sd, double cd) {
  return -(r[0] * cd * cp + r[1] * cd * sp + r[2] * sd) * kInvClight;
}

// arrival-time offset relative to the geocentre, -r . n / c
MBIS_HD double geocentre_delay(const double* r, double ra, double dec, double gmst) {
  const double ph = ra - gmst, cd = cos(dec);
  return -(r[0] * cd * cos(ph) + r[1] * cd * sin(ph) + r[2] * sin(dec)) * kInvClight;
}

}  // namespace mbis
