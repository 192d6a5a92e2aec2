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
// as an online log-sum-exp: in FP64 in log_distance_marginal (the FP64 path), in FP32 about
// an FP64 reference value in log_distance_marginal_mixed (the mixed-precision kernels).
#pragma once
#include "physics.cuh"

namespace mbis {

// Gauss-Legendre nodes/weights on [-1, 1]: x48, w48, x8, w8 (host fills, device reads)
constexpr int kGL48 = 48, kGL8 = 8;
// a range of the mixed-precision distance rule whose largest log-integrand lies this far below
// the window's is left out
constexpr float kDistSkip = 45.0f;
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

// ln I0(x) - x in FP32 (x >= 0), slowly varying, so FP32 keeps its absolute accuracy.  The
// polynomial approximations of Abramowitz & Stegun 9.8.1 (x < 3.75: I0 in (x/3.75)^2) and
// 9.8.2 (x >= 3.75: x^(1/2) e^(-x) I0(x) in 3.75/x) give |error| < 5e-7 in the logarithm
// over all x >= 0, with one fast logarithm and no division.
__device__ __forceinline__ float log_i0_minus_x_f(float x) {
  if (x < 3.75f) {
    const float t = x * x * (1.0f / 14.0625f);
    const float p =
        fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, 0.0045813f, 0.0360768f), 0.2659732f), 1.2067492f), 3.0899424f),
                     3.5156229f),
             1.0f);
    return __logf(p) - x;
  }
  const float t = __fdividef(3.75f, x);
  const float p = fmaf(
      t,
      fmaf(t,
           fmaf(t,
                fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, 0.00392377f, -0.01647633f), 0.02635537f), -0.02057706f),
                             0.00916281f),
                     -0.00157565f),
                0.00225319f),
           0.01328592f),
      0.39894228f);
  return __logf(p * rsqrtf(x));
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

// G(s) - G(s_ref) at the offset d = s - s_ref, in FP32: u - u_ref = u_ref expm1(d) keeps the
// differences small, so FP32 carries ~1e-6 relative accuracy on each weight.
__device__ __forceinline__ float dist_node_g(float d, float Z, float H, float u_ref, float phi_ref) {
  const float du = u_ref * expm1f(d);
  const float u = u_ref + du;
  return Z * du - 0.5f * H * du * (2.0f * u_ref + du) - 3.0f * d + (log_i0_minus_x_f(Z * u) - phi_ref);
}

// One composite rule over [lo, hi] (offsets from the reference point s_ref).
__device__ __forceinline__ void dist_rule_f(LogSumExpF& L, float lo, float hi, int panels, int n, const float* x,
                                            const float* w, float Z, float H, float u_ref, float phi_ref) {
  const float h = (hi - lo) * (1.0f / (float)panels), half = 0.5f * h;
  for (int p = 0; p < panels; ++p) {
    const float mid = fmaf((float)p + 0.5f, h, lo);
    for (int i = 0; i < n; ++i) L.add(dist_node_g(fmaf(half, __ldg(x + i), mid), Z, H, u_ref, phi_ref), half * __ldg(w + i));
  }
}
#endif

// Per-context constants of the distance marginal: c0 = ln(3 / (dmax^3 - dmin^3)), the
// large-distance end u_lo = 1 / dmax rounded to FP32 with s_lo = ln(u_lo) taken from that
// rounded value (so that the FP32 reference points below stay consistent with their
// logarithms), and the width of the range in s.
struct DistConst {
  double c0, s_lo;
  float u_lo, span;
};

inline DistConst dist_const(double dmin, double dmax) {
  DistConst d;
  d.c0 = std::log(3.0 / (dmax * dmax * dmax - dmin * dmin * dmin));
  d.u_lo = (float)(1.0 / dmax);
  d.s_lo = std::log((double)d.u_lo);
  d.span = (float)(-std::log(dmin) - d.s_lo);
  return d;
}

#ifdef __CUDACC__
// The distance marginal of log_distance_marginal with the same rules (48-point window of
// +-12 widths about the peak, 4-panel 8-point composite rules outside it; 24 panels of 8
// points without a peak), taken in FP32 about a reference point s_ref (the peak, or the
// large-distance end): every node contributes G(s) - G(s_ref) from dist_rule_f, and G(s_ref)
// itself is assembled in FP64 from exact products,
//   G(s_ref) = c0 - 3 s_ref + Z u_ref + [ln I0(Z u_ref) - Z u_ref] - H u_ref^2 / 2,
// so that the few terms that grow with the signal (Z u_ref, H u_ref^2 reach 10^4) keep FP64
// accuracy while the bracket, the window and the nodes run in FP32.  The reference u_ref is
// an FP32 number and s_ref = s_lo + (its offset), consistent with ln u_ref to FP32 rounding.
__device__ __forceinline__ double log_distance_marginal_mixed(double Z, double H, const DistConst& dc,
                                                              const float* gl) {
  const float* x48 = gl;
  const float* w48 = gl + kGL48;
  const float* x8 = gl + 2 * kGL48;
  const float* w8 = gl + 2 * kGL48 + kGL8;
  const float Zf = (float)Z, Hf = (float)H, span = dc.span;
  bool window = false;
  float wlo = 0.0f, whi = span, r_ref = 0.0f;  // offsets from s_lo
  if (Hf > 0.0f && Zf * Zf > 14.0f * Hf) {
    const float u = (Zf + sqrtf(Zf * Zf - 14.0f * Hf)) / (2.0f * Hf);
    const float sig = rsqrtf(fmaxf(Zf * u - 7.0f, 1e-30f));
    const float rc = logf(u / dc.u_lo);
    wlo = fmaxf(0.0f, rc - 12.0f * sig);
    whi = fminf(span, rc + 12.0f * sig);
    window = wlo < whi;
    r_ref = fminf(fmaxf(rc, 0.0f), span);
  }
  const float uf = dc.u_lo * __expf(r_ref);
  const float phi_ref = log_i0_minus_x_f(Zf * uf);
  LogSumExpF L;
  if (window) {
    dist_rule_f(L, wlo - r_ref, whi - r_ref, 1, kGL48, x48, w48, Zf, Hf, uf, phi_ref);
    // Outside the window: G has at most one local maximum (G' = f(x) - 3 with
    // f(x) = x I1(x)/I0(x) - (H/Z^2) x^2 rising then falling in x = Z e^s), so a range that
    // does not hold it takes its largest value at its ends.  A range whose ends lie more than
    // kDistSkip below the window's largest node is left out: its share of the integral is
    // below e^-40.  (Were the maximum inside the range, the window's nearest end would be
    // within kDistSkip of the window's largest node and the range would be summed.)
    if (wlo > 0.0f) {
      const float g_end = fmaxf(dist_node_g(-r_ref, Zf, Hf, uf, phi_ref), dist_node_g(wlo - r_ref, Zf, Hf, uf, phi_ref));
      if (g_end > L.m - kDistSkip) dist_rule_f(L, -r_ref, wlo - r_ref, 4, kGL8, x8, w8, Zf, Hf, uf, phi_ref);
    }
    if (whi < span && dist_node_g(whi - r_ref, Zf, Hf, uf, phi_ref) > L.m - kDistSkip)
      dist_rule_f(L, whi - r_ref, span - r_ref, 4, kGL8, x8, w8, Zf, Hf, uf, phi_ref);
  } else {
    dist_rule_f(L, -r_ref, span - r_ref, 24, kGL8, x8, w8, Zf, Hf, uf, phi_ref);
  }
  const double u_ref = (double)uf;
  const double g_ref = dc.c0 - 3.0 * (dc.s_lo + (double)r_ref) + Z * u_ref - 0.5 * H * u_ref * u_ref + (double)phi_ref;
  return g_ref + (double)L.m + (double)logf(L.acc);
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

// the same table rounded to FP32 (the mixed-precision marginal's copy)
inline void fill_gauss_legendre_f32(float* glf) {
  double gl[kGLSize];
  fill_gauss_legendre(gl);
  for (int i = 0; i < kGLSize; ++i) glf[i] = (float)gl[i];
}

}  // namespace mbis
