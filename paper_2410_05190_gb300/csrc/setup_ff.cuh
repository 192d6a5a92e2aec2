// setup_ff.cuh -- the per-sample set-up of the time-marginalised kernel (sample_setup in
// physics.cuh: amplitude, TaylorF2 phase coefficients, ISCO cut) in float-float arithmetic.
// The same series and the same Newton-refined powers; every value to ~1e-14 relative, with
// one FP64 logarithm (ln pi M) and a handful of FP64 operations where a double is the input
// or the output.  The GB300 runs FP64 at a small fraction of its FP32 rate.
#pragma once
#include "ffloat.cuh"
#include "physics.cuh"

namespace mbis {

__device__ __forceinline__ FF ffk(const FFConst k) { return FF{k.h, k.l}; }
__device__ __forceinline__ FF ffs(float x) { return FF{x, 0.f}; }

// 1 / x from an FP32 reciprocal and one Newton step in float-float
__device__ __forceinline__ FF ff_rcp(FF x) {
  const float r0 = __frcp_rn(x.h);
  const FF e = ff_add_f(ff_neg(ff_mul(x, ffs(r0))), 1.0f);  // 1 - x r0, ~2^-24
  return ff_add(ffs(r0), ff_mul(ffs(r0), e));
}

// The PN factors of pn_terms (physics.cuh) in float-float
__device__ __forceinline__ void pn_terms_ff(FF eta, FF dm, FF xs, FF xa, FF (&t)[6]) {
  const FF e2 = ff_mul(eta, eta), e3 = ff_mul(e2, eta);
  const FF dxa = ff_mul(dm, xa), xa2 = ff_mul(xa, xa), xs2 = ff_mul(xs, xs), dxaxs = ff_mul(dxa, xs);
  constexpr double kLn4 = 1.3862943611198906188344642429164;
  constexpr double pi2 = kPi * kPi;
  // phi2
  t[0] = ff_add(ffk(FFConst(3715.0 / 756.0)), ff_mul(ffk(FFConst(55.0 / 9.0)), eta));
  // phi3
  t[1] = ff_add(ff_add(ffk(FFConst(-16.0 * kPi)), ff_mul(ffk(FFConst(113.0 / 3.0)), dxa)),
                ff_mul(ff_add(ffk(FFConst(113.0 / 3.0)), ff_mul(ffk(FFConst(-76.0 / 3.0)), eta)), xs));
  // phi4
  {
    FF v = ff_add(ffk(FFConst(15293365.0 / 508032.0)), ff_mul(ffk(FFConst(27145.0 / 504.0)), eta));
    v = ff_add(v, ff_mul(ffk(FFConst(3085.0 / 72.0)), e2));
    v = ff_add(v, ff_mul(ff_add(ffk(FFConst(-405.0 / 8.0)), ff_mul(ffk(FFConst(200.0)), eta)), xa2));
    v = ff_add(v, ff_mul(ffk(FFConst(-405.0 / 4.0)), dxaxs));
    v = ff_add(v, ff_mul(ff_add(ffk(FFConst(-405.0 / 8.0)), ff_mul(ffk(FFConst(5.0 / 2.0)), eta)), xs2));
    t[2] = v;
  }
  // c5 (phi5 = c5 (1 + 3 ln v))
  {
    FF v = ff_add(ffk(FFConst(kPi * 38645.0 / 756.0)), ff_mul(ffk(FFConst(-kPi * 65.0 / 9.0)), eta));
    v = ff_add(v, ff_mul(ff_add(ffk(FFConst(-732985.0 / 2268.0)), ff_mul(ffk(FFConst(-140.0 / 9.0)), eta)), dxa));
    FF s = ff_add(ffk(FFConst(-732985.0 / 2268.0)), ff_mul(ffk(FFConst(24260.0 / 81.0)), eta));
    s = ff_add(s, ff_mul(ffk(FFConst(340.0 / 9.0)), e2));
    t[3] = ff_add(v, ff_mul(s, xs));
  }
  // a6 (phi6 = a6 - 6848/21 ln v)
  {
    FF v = ffk(FFConst(11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 - 6848.0 / 21.0 * (kEulerGamma + kLn4)));
    v = ff_add(v, ff_mul(ffk(FFConst(-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2)), eta));
    v = ff_add(v, ff_mul(ffk(FFConst(76055.0 / 1728.0)), e2));
    v = ff_add(v, ff_mul(ffk(FFConst(-127825.0 / 1296.0)), e3));
    v = ff_add(v, ff_mul(ffk(FFConst(kPi * 2270.0 / 3.0)), dxa));
    v = ff_add(v, ff_mul(ff_add(ffk(FFConst(kPi * 2270.0 / 3.0)), ff_mul(ffk(FFConst(-520.0 * kPi)), eta)), xs));
    v = ff_add(v, ff_mul(ff_add(ffk(FFConst(75515.0 / 144.0)), ff_mul(ffk(FFConst(-8225.0 / 18.0)), eta)), dxaxs));
    FF sa = ff_add(ffk(FFConst(75515.0 / 288.0)), ff_mul(ffk(FFConst(-263245.0 / 252.0)), eta));
    sa = ff_add(sa, ff_mul(ffk(FFConst(-480.0)), e2));
    v = ff_add(v, ff_mul(sa, xa2));
    FF ss = ff_add(ffk(FFConst(75515.0 / 288.0)), ff_mul(ffk(FFConst(-232415.0 / 504.0)), eta));
    ss = ff_add(ss, ff_mul(ffk(FFConst(1255.0 / 9.0)), e2));
    t[4] = ff_add(v, ff_mul(ss, xs2));
  }
  // phi7
  {
    FF v = ff_add(ffk(FFConst(kPi * 77096675.0 / 254016.0)), ff_mul(ffk(FFConst(kPi * 378515.0 / 1512.0)), eta));
    v = ff_add(v, ff_mul(ffk(FFConst(-kPi * 74045.0 / 756.0)), e2));
    FF s = ff_add(ffk(FFConst(-25150083775.0 / 3048192.0)), ff_mul(ffk(FFConst(10566655595.0 / 762048.0)), eta));
    s = ff_add(s, ff_mul(ffk(FFConst(-1042165.0 / 3024.0)), e2));
    s = ff_add(s, ff_mul(ffk(FFConst(5345.0 / 36.0)), e3));
    v = ff_add(v, ff_mul(s, xs));
    FF d = ff_add(ffk(FFConst(-25150083775.0 / 3048192.0)), ff_mul(ffk(FFConst(26804935.0 / 6048.0)), eta));
    d = ff_add(d, ff_mul(ffk(FFConst(-1985.0 / 48.0)), e2));
    t[5] = ff_add(v, ff_mul(d, dxa));
  }
}

struct SampleSetupFF {
  FF C[kNumBasis];  // phase coefficients (turns), as sample_setup's pc.C
  FF cst;
  double amp;       // A at d_L = dl_mpc
  int32_t kcut;     // grid points f_lo + k df strictly below the ISCO
};

// sample_setup in float-float: M = Mc T_sun u^(3/5) (u = 1/eta), a = pi M with a^(1/3) and
// 1/a; y^5 = u^3, c^3 = a and z^6 = x^5 (x = Mc T_sun) each one Newton step from an FP32
// seed, the step's small numerator taken in float-float; ln a in FP64.
__device__ __forceinline__ SampleSetupFF sample_setup_ff(double mc_d, double q_d, double chi1, double chi2,
                                                         double tc, double phic, double dl_mpc, double f_lo,
                                                         double df, int32_t n_bins) {
  SampleSetupFF o;
  const FF q = ff_from_double(q_d), mc = ff_from_double(mc_d);
  const FF w = ff_rcp(ff_add_f(q, 1.0f));
  const FF u = ff_add(ff_add_f(q, 2.0f), ff_rcp(q));
  const FF eta = ff_mul(q, ff_mul(w, w)), dm = ff_mul(ff_add_f(q, -1.0f), w);
  FF y;
  {
    const float y0 = powf(u.h, 0.6f);
    const FF y2 = ff_mul(ffs(y0), ffs(y0)), y4 = ff_mul(y2, y2);
    const FF f = ff_sub(ff_mul(y4, ffs(y0)), ff_mul(ff_mul(u, u), u));  // y0^5 - u^3
    y = ff_add_f(ffs(y0), -f.h * __frcp_rn(5.0f * y4.h));
  }
  const FF a = ff_mul(ff_mul(ffk(FFConst(kPi * kTsun)), mc), y);
  const double la_d = log(ff_to_double(a));
  const FF la = ff_from_double(la_d);
  FF a13;
  {
    const float c0 = cbrtf(a.h);
    const FF f = ff_sub(ff_mul(ff_mul(ffs(c0), ffs(c0)), ffs(c0)), a);  // c0^3 - a
    a13 = ff_add_f(ffs(c0), -f.h * __frcp_rn(3.0f * c0 * c0));
  }
  const FF a23 = ff_mul(a13, a13), inv_a = ff_rcp(a);
  {
    const FF x = ff_mul(mc, ffk(FFConst(kTsun)));
    const FF x2 = ff_mul(x, x), x5 = ff_mul(ff_mul(x2, x2), x);
    const float z0 = powf(x.h, 5.0f / 6.0f);
    const FF z2 = ff_mul(ffs(z0), ffs(z0)), z4 = ff_mul(z2, z2);
    const FF f = ff_sub(ff_mul(z4, z2), x5);  // z0^6 - x^5
    const FF z = ff_add_f(ffs(z0), -f.h * __frcp_rn(6.0f * z4.h * z0));
    const FF inv_d = ff_rcp(ff_mul(ff_from_double(dl_mpc), ffk(FFConst(kMpcSeconds))));
    o.amp = ff_to_double(ff_mul(ff_mul(ffk(FFConst(0.45643546458763845 * 0.46619407703541166)), z), inv_d));
  }
  FF t[6];
  pn_terms_ff(eta, dm, ff_from_double(0.5 * (chi1 + chi2)), ff_from_double(0.5 * (chi1 - chi2)), t);
  const FF pre = ff_mul(ffk(FFConst(3.0 / (256.0 * kPi))), u);  // 3 / (128 eta) / (2 pi), turns
  const FF pa = ff_mul(pre, inv_a), pa13 = ff_mul(pre, a13);
  o.C[0] = ff_mul(ff_mul(pa, inv_a), a13);                 // a^(-5/3)
  o.C[1] = ff_mul(pa, t[0]);                               // a^(-1)
  o.C[2] = ff_mul(ff_mul(pa, t[1]), a13);                  // a^(-2/3)
  o.C[3] = ff_mul(ff_mul(pa, t[2]), a23);                  // a^(-1/3)
  o.C[4] = ff_mul(pre, t[3]);                              // ln f
  o.C[5] = ff_mul(pa13, ff_sub(t[4], ff_mul(ffk(FFConst(6848.0 / 63.0)), la)));
  o.C[6] = ff_mul(pa13, ffk(FFConst(-6848.0 / 63.0)));
  o.C[7] = ff_mul(ff_mul(pre, t[5]), a23);
  o.C[8] = ff_from_double(tc);
  o.cst = ff_add(ff_add_f(ff_mul(ff_from_double(phic), ffk(FFConst(-1.0 / kTwoPi))), -0.125f),
                 ff_mul(ff_mul(pre, t[3]), ff_add_f(la, 1.0f)));

  // the cut: an FP32 estimate of ceil((f_isco - f_lo) / df), then exact FP64 steps to the
  // first grid point at or above f_isco
  const double fi = ff_to_double(ff_mul(inv_a, ffk(FFConst(1.0 / 14.696938456699067))));
  const float kf = ceilf((float)(fi - f_lo) * __frcp_rn((float)df));
  int32_t k = !(kf > 0.0f) ? 0 : (kf >= (float)n_bins ? n_bins : (int32_t)kf);
  while (k > 0 && f_lo + (double)(k - 1) * df >= fi) --k;
  while (k < n_bins && f_lo + (double)k * df < fi) ++k;
  o.kcut = k;
  return o;
}

}  // namespace mbis
