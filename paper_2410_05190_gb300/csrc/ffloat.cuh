// ffloat.cuh -- float-float ("double-single") helpers for the anchor-block entry of the
// mixed-precision kernels, for events whose phase terms stay below kFloatFloatMaxTurns, and
// for their running sums of FP32 partial sums.
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

}  // namespace mbis
