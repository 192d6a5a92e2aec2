// anchor.cuh -- device reads of an anchor block (internal.h, AnchorBlock) shared by the
// mixed-precision likelihood kernels: the coefficients of the FP32 remainder polynomial
// of a sample on the block, from the block's remainder table read as 16-byte vectors.
#pragma once
#include "internal.h"

namespace mbis {

// c[m] = sum_j cf(j) E[j][m] for m = 0..D, the sum taken over j = 0..7 in order (FMA into
// zero).  E is [8][6] floats: two rows are three 16-byte vectors.
template <int D, typename CF>
__device__ __forceinline__ void remainder_coeffs(const AnchorBlock& B, CF cf, float (&c)[D + 1]) {
  static_assert(kRemDegMax + 1 == 6 && D <= kRemDegMax, "two remainder rows per three vectors");
  const float4* ev = reinterpret_cast<const float4*>(&B.E[0][0]);
#pragma unroll
  for (int m = 0; m <= D; ++m) c[m] = 0.f;
#pragma unroll
  for (int p = 0; p < (kNumBasis - 1) / 2; ++p) {
    const float4 e0 = __ldg(ev + 3 * p), e1 = __ldg(ev + 3 * p + 1), e2 = __ldg(ev + 3 * p + 2);
    const float ra[6] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y};  // E[2p][0..5]
    const float rb[6] = {e1.z, e1.w, e2.x, e2.y, e2.z, e2.w};  // E[2p + 1][0..5]
    const float ca = cf(2 * p), cb = cf(2 * p + 1);
#pragma unroll
    for (int m = 0; m <= D; ++m) c[m] = fmaf(ca, ra[m], c[m]);
#pragma unroll
    for (int m = 0; m <= D; ++m) c[m] = fmaf(cb, rb[m], c[m]);
  }
}

}  // namespace mbis
