// marg.cuh -- analytic phase and numeric distance marginalisation (Sec. III: the
// likelihood is marginalised over phase and distance with analytic / numeric formulas).
//
// Phase: a uniform phi_c turns exp(Re(e^(i phi_c) Z)) into I0(|Z|).
// Distance: with Z1, H1 the overlap and norm at d_L = 1 Mpc, Z = Z1/d and H = H1/d^2, and
//   L(d) = I0(Z1/d) exp(-H1/(2 d^2)),  p(d) = 3 d^2 / (dmax^3 - dmin^3) on [dmin, dmax].
// The integral is taken in s = ln(1/d), where the integrand
//   G(s) = ln(3/(dmax^3 - dmin^3)) - 3 s + ln I0(Z1 e^s) - H1 e^(2s) / 2
// has, for a loud match (Z1^2 > 14 H1), a peak at u = e^s solving H1 u^2 - Z1 u + 7/2 = 0
// (large-argument I1/I0 ~ 1 - 1/(2x)) of width 1/sqrt(Z1 u - 7).  A 48-point Gauss-Legendre
// rule covers +-12 widths about the peak and 8-point composite rules the rest of the
// range; without a peak the whole range gets a 24-panel composite 8-point rule.  Sums run
// as an online log-sum-exp in FP64.
#pragma once
#include "physics.cuh"

namespace mbis {

// Gauss-Legendre nodes/weights on [-1, 1]: x48, w48, x8, w8 (host fills, device reads)
constexpr int kGL48 = 48, kGL8 = 8;
constexpr int kGLSize = 2 * kGL48 + 2 * kGL8;

#ifdef __CUDACC__
__device__ __forceinline__ double log_i0(double x) {
  x = fabs(x);
  if (x < 700.0) return log(cyl_bessel_i0(x));
  // Hankel expansion e^x / sqrt(2 pi x) * sum_k ((2k-1)!!)^2 / (k! (8x)^k)
  const double t = 1.0 / (8.0 * x);
  const double s = 1.0 + t * (1.0 + t * (4.5 + t * (37.5 + t * 459.375)));
  return x - 0.5 * log(kTwoPi * x) + log(s);
}

struct LogSumExp {
  double m = -INFINITY, acc = 0.0;
  __device__ __forceinline__ void add(double g, double w) {
    if (g > m) {
      acc = acc * exp(m - g) + w;
      m = g;
    } else {
      acc += w * exp(g - m);
    }
  }
  __device__ __forceinline__ double value() const { return m + log(acc); }
};

__device__ __forceinline__ void dist_rule(LogSumExp& L, double a, double b, int panels, int n, const double* x,
                                          const double* w, double Z, double H, double c0) {
  const double h = (b - a) / panels;
  for (int p = 0; p < panels; ++p) {
    const double mid = a + (p + 0.5) * h, half = 0.5 * h;
    for (int i = 0; i < n; ++i) {
      const double s = mid + half * x[i];
      const double u = exp(s);
      const double g = c0 - 3.0 * s + log_i0(Z * u) - 0.5 * H * u * u;
      L.add(g, half * w[i]);
    }
  }
}

__device__ __forceinline__ double log_distance_marginal(double Z, double H, double dmin, double dmax,
                                                        const double* gl) {
  const double* x48 = gl;
  const double* w48 = gl + kGL48;
  const double* x8 = gl + 2 * kGL48;
  const double* w8 = gl + 2 * kGL48 + kGL8;
  const double c0 = log(3.0 / (dmax * dmax * dmax - dmin * dmin * dmin));
  const double s_lo = -log(dmax), s_hi = -log(dmin);
  LogSumExp L;
  bool window = false;
  double wlo = s_lo, whi = s_hi;
  if (H > 0.0 && Z * Z > 14.0 * H) {
    const double u = (Z + sqrt(Z * Z - 14.0 * H)) / (2.0 * H);
    const double sig = 1.0 / sqrt(fmax(Z * u - 7.0, 1e-300));
    const double sc = log(u);
    wlo = fmax(s_lo, sc - 12.0 * sig);
    whi = fmin(s_hi, sc + 12.0 * sig);
    window = wlo < whi;
  }
  if (window) {
    dist_rule(L, wlo, whi, 1, kGL48, x48, w48, Z, H, c0);
    if (wlo > s_lo) dist_rule(L, s_lo, wlo, 8, kGL8, x8, w8, Z, H, c0);
    if (whi < s_hi) dist_rule(L, whi, s_hi, 8, kGL8, x8, w8, Z, H, c0);
  } else {
    dist_rule(L, s_lo, s_hi, 24, kGL8, x8, w8, Z, H, c0);
  }
  return L.value();
}

// ln I0(x) - x in FP32 (x >= 0): slowly varying, so FP32 keeps its absolute accuracy
__device__ __forceinline__ float log_i0_minus_x_f(float x) {
  if (x < 15.0f) return logf(cyl_bessel_i0f(x)) - x;
  const float t = 1.0f / (8.0f * x);
  const float s = t * (1.0f + t * (4.5f + t * (37.5f + t * 459.375f)));
  return -0.5f * logf(6.28318530717958647692f * x) + log1pf(s);
}

struct LogSumExpF {
  float m = -INFINITY, acc = 0.0f;
  __device__ __forceinline__ void add(float g, float w) {
    if (g > m) {
      acc = acc * __expf(m - g) + w;
      m = g;
    } else {
      acc += w * __expf(g - m);
    }
  }
};

// The same quadrature as log_distance_marginal, with the nodes evaluated in FP32 as
// differences G(s) - G(s_ref) from one FP64 evaluation at s_ref (the peak, or the
// large-distance end when there is none).  The differences are formed from small
// quantities (u - u_ref = u_ref expm1(s - s_ref)), so FP32 keeps ~1e-6 relative accuracy
// on each weight and the result carries the FP64 accuracy of G(s_ref).
__device__ __forceinline__ void dist_rule_f(LogSumExpF& L, double a, double b, int panels, int n, const double* x,
                                            const double* w, float Z, float H, double s_ref, float u_ref,
                                            float phi_ref) {
  const double h = (b - a) / panels;
  for (int p = 0; p < panels; ++p) {
    const double mid = a + (p + 0.5) * h;
    const float half = (float)(0.5 * h);
    const float dmid = (float)(mid - s_ref);
    for (int i = 0; i < n; ++i) {
      const float d = fmaf(half, (float)x[i], dmid);  // s - s_ref
      const float du = u_ref * expm1f(d);
      const float u = u_ref + du;
      const float g = Z * du - 0.5f * H * du * (2.0f * u_ref + du) - 3.0f * d + (log_i0_minus_x_f(Z * u) - phi_ref);
      L.add(g, half * (float)w[i]);
    }
  }
}

__device__ __forceinline__ double log_distance_marginal_mixed(double Z, double H, double dmin, double dmax,
                                                              const double* gl) {
  const double* x48 = gl;
  const double* w48 = gl + kGL48;
  const double* x8 = gl + 2 * kGL48;
  const double* w8 = gl + 2 * kGL48 + kGL8;
  const double c0 = log(3.0 / (dmax * dmax * dmax - dmin * dmin * dmin));
  const double s_lo = -log(dmax), s_hi = -log(dmin);
  bool window = false;
  double wlo = s_lo, whi = s_hi, s_ref = s_lo;
  if (H > 0.0 && Z * Z > 14.0 * H) {
    const double u = (Z + sqrt(Z * Z - 14.0 * H)) / (2.0 * H);
    const double sig = 1.0 / sqrt(fmax(Z * u - 7.0, 1e-300));
    const double sc = log(u);
    wlo = fmax(s_lo, sc - 12.0 * sig);
    whi = fmin(s_hi, sc + 12.0 * sig);
    window = wlo < whi;
    s_ref = fmin(fmax(sc, s_lo), s_hi);
  }
  const double u_ref = exp(s_ref);
  const double g_ref = c0 - 3.0 * s_ref + log_i0(Z * u_ref) - 0.5 * H * u_ref * u_ref;
  const float Zf = (float)Z, Hf = (float)H, uf = (float)u_ref;
  const float phi_ref = log_i0_minus_x_f(Zf * uf);
  LogSumExpF L;
  if (window) {
    dist_rule_f(L, wlo, whi, 1, kGL48, x48, w48, Zf, Hf, s_ref, uf, phi_ref);
    if (wlo > s_lo) dist_rule_f(L, s_lo, wlo, 4, kGL8, x8, w8, Zf, Hf, s_ref, uf, phi_ref);
    if (whi < s_hi) dist_rule_f(L, whi, s_hi, 4, kGL8, x8, w8, Zf, Hf, s_ref, uf, phi_ref);
  } else {
    dist_rule_f(L, s_lo, s_hi, 24, kGL8, x8, w8, Zf, Hf, s_ref, uf, phi_ref);
  }
  return g_ref + (double)L.m + log((double)L.acc);
}
#endif

// host: Gauss-Legendre nodes by Newton iteration on the Legendre recurrence
inline void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

inline void fill_gauss_legendre(double* gl) {
  gauss_legendre(kGL48, gl, gl + kGL48);
  gauss_legendre(kGL8, gl + 2 * kGL48, gl + 2 * kGL48 + kGL8);
}

}  // namespace mbis
