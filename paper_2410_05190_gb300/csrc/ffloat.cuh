// ffloat.cuh -- float-float ("double-single") helpers: the anchor-block entry of the
// mixed-precision kernels (events whose phase terms stay below kFloatFloatMaxTurns), their
// running sums of FP32 partial sums, and the per-sample set-up of the time-marginalised
// kernel (pair arithmetic, sine and cosine, a 64-bit turn fraction).
#pragma once
#include <cstdint>

namespace mbis {

// A value is an unevaluated pair hi + lo of floats.  Sums use Knuth's two-sum (exact), the
// product of a pair by a pair Dekker's product with the FMA giving the rounding error of
// hi*hi exactly; explicit _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A running sum of floats as an unevaluated pair: each addition into h is error-free
// (two-sum) and its rounding error is gathered in l, so the pair carries ~2^-48 relative
// accuracy without FP64 arithmetic (which the GB300 runs at a small fraction of FP32).
struct FFSum {
  float h = 0.0f, l = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(h, x, s, e);
    h = s;
    l = __fadd_rn(l, e);
  }
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};

// (sh, sl) += (ch, cl) * (bh, bl)
__device__ __forceinline__ void ff_mac(float ch, float cl, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ch, bh);
  const float e = __fmaf_rn(ch, bl, __fmaf_rn(cl, bh, __fmaf_rn(ch, bh, -p)));
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// frac(h + l) as a 32-bit fixed-point turn count (|h| < 2^31 turns); resid (turns) is what
// the count rounds off.  h 2^32 and l 2^32 are exact scalings; their integer parts are taken
// modulo 2^32 through a 64-bit conversion (a frac() taken first would round for h < 0).
__device__ __forceinline__ uint32_t ff_frac32(float h, float l, float& resid) {
  const float xh = __fmul_rn(h, 4294967296.0f), xl = __fmul_rn(l, 4294967296.0f);
  const float rh = rintf(xh), rl = rintf(xl);
  resid = __fmul_rn(__fadd_rn(__fsub_rn(xh, rh), __fsub_rn(xl, rl)), 2.3283064365386963e-10f);
  return (uint32_t)(unsigned long long)__float2ll_rn(rh) + (uint32_t)__float2int_rn(rl);
}

// ---- pairs as values: a few operations of float-float arithmetic -----------------------
struct FF {
  float h, l;
};

// (a, b) with |a| >= |b| as a normalised pair (fast two-sum)
__device__ __forceinline__ FF ff_renorm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ff_renorm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
  return ff_renorm(p, e);
}

// a + b for a float b
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  return ff_renorm(s, __fadd_rn(e, a.l));
}

__device__ __forceinline__ FF ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return FF{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.h + (double)a.l; }

// a constant as a pair, split at compile time
struct FFConst {
  float h, l;
  __host__ __device__ constexpr explicit FFConst(double c) : h((float)c), l((float)(c - (double)(float)c)) {}
};

// Sine and cosine of an FP64 angle |x| < 2^20 as float-float pairs, with an absolute error
// below ~1e-13 for |x| < 8 pi (beyond, the FP64 pi/2 adds |k| 6e-17): a Cody-Waite
// reduction x = k pi/2 + r (k = rint(2x/pi) from an FP32 estimate, r by one FP64 fused
// multiply-add: |r| <= pi/4 plus the estimate's error), then the Taylor series of sin r and
// cos r, which at |r| <= 0.79 leave out less than r^15/15! = 2e-14 and r^16/16! = 1e-15.  The terms below ~2e-7 (r^11 and up, r^10 and up) are summed in FP32;
// the others in float-float.  Two FP64 operations and three conversions per call, against
// several tens on the FP64 pipe for the library's double-precision sincos, which the GB300
// runs at a small fraction of FP32.
__device__ __forceinline__ void ff_sincos(double x, FF& s_out, FF& c_out) {
  constexpr double kPiO2 = 1.5707963267948966192313216916398;
  const float kf = rintf(__fmul_rn(__double2float_rn(x), 0.63661977236758134f));
  const double r = fma(-(double)kf, kPiO2, x);
  const FF rr = ff_from_double(r);
  const FF r2 = ff_mul(rr, rr);
  const float z = r2.h;
  // sin r = r (1 + z (-1/3! + z (1/5! + z (-1/7! + z (1/9! + z t))))), t = -1/11! + z/13!
  float t = __fmaf_rn(z, 1.6059043836821614e-10f, -2.5052108385441720e-8f);
  FF p;
  {
    constexpr FFConst c9(1.0 / 362880.0), c7(-1.0 / 5040.0), c5(1.0 / 120.0), c3(-1.0 / 6.0);
    p = ff_add(FF{c9.h, c9.l}, FF{__fmul_rn(z, t), 0.0f});
    p = ff_add(FF{c7.h, c7.l}, ff_mul(r2, p));
    p = ff_add(FF{c5.h, c5.l}, ff_mul(r2, p));
    p = ff_add(FF{c3.h, c3.l}, ff_mul(r2, p));
    p = ff_add_f(ff_mul(r2, p), 1.0f);
  }
  const FF sn = ff_mul(rr, p);
  // cos r = 1 + z (-1/2! + z (1/4! + z (-1/6! + z (1/8! + z u)))), u = -1/10! + z (1/12! - z/14!)
  float u = __fmaf_rn(z, -1.1470745597729725e-11f, 2.0876756987868099e-9f);
  u = __fmaf_rn(z, u, -2.7557319223985891e-7f);
  FF q;
  {
    constexpr FFConst c8(1.0 / 40320.0), c6(-1.0 / 720.0), c4(1.0 / 24.0), c2(-0.5);
    q = ff_add(FF{c8.h, c8.l}, FF{__fmul_rn(z, u), 0.0f});
    q = ff_add(FF{c6.h, c6.l}, ff_mul(r2, q));
    q = ff_add(FF{c4.h, c4.l}, ff_mul(r2, q));
    q = ff_add(FF{c2.h, c2.l}, ff_mul(r2, q));
    q = ff_add_f(ff_mul(r2, q), 1.0f);
  }
  const FF cs = q;
  // quadrant k mod 4: (sin, cos) of r + k pi/2
  const int k = (int)kf & 3;
  const FF msn = FF{-sn.h, -sn.l}, mcs = FF{-cs.h, -cs.l};
  s_out = k == 0 ? sn : (k == 1 ? cs : (k == 2 ? msn : mcs));
  c_out = k == 0 ? cs : (k == 1 ? msn : (k == 2 ? mcs : sn));
}

// Any FP64 angle: an angle beyond the reduction's range takes the library's sincos
__device__ __forceinline__ void ff_sincos_any(double x, FF& s, FF& c) {
  if (fabs(x) < 1048576.0) {
    ff_sincos(x, s, c);
  } else {
    double sd, cd;
    sincos(x, &sd, &cd);
    s = ff_from_double(sd);
    c = ff_from_double(cd);
  }
}

// The same as FP64 values
__device__ __forceinline__ void ff_sincos_d(double x, double& s, double& c) {
  FF fs, fc;
  ff_sincos_any(x, fs, fc);
  s = ff_to_double(fs);
  c = ff_to_double(fc);
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.h, -a.l}; }
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }

// frac(h + l) as a 64-bit fixed-point turn count (|h| < 256 turns): the integer parts of
// h 2^32 and l 2^32 give the upper word modulo 2^32, their fractional parts (exact) the
// lower word, rounded at 2^-56 turns; a negative lower word borrows from the upper one.
__device__ __forceinline__ uint64_t ff_frac64(FF v) {
  const float xh = __fmul_rn(v.h, 4294967296.0f), xl = __fmul_rn(v.l, 4294967296.0f);
  const float rh = rintf(xh), rl = rintf(xl);
  const float f = __fadd_rn(__fsub_rn(xh, rh), __fsub_rn(xl, rl));  // in [-1, 1] units of 2^-32
  const uint32_t hi = (uint32_t)(unsigned long long)__float2ll_rn(rh) + (uint32_t)__float2int_rn(rl);
  return ((uint64_t)hi << 32) + (uint64_t)__float2ll_rn(__fmul_rn(f, 4294967296.0f));
}

}  // namespace mbis
