// k_draw.cu -- proposal draws (g of Eq. 5) and prior densities (pi of Eq. 5).
//
// One thread per sample.  Normals come from Philox4x32-10 (philox.cuh).  Sample i of a
// call uses counter (lo32(ctr0 + i), hi32(ctr0 + i), 2, block) and key (lo32(seed),
// hi32(seed)); each block yields two Box-Muller pairs.  Because the counter names the
// sample, a sample's value does not depend on batch boundaries, launch shape or scheduling.
#include "internal.h"
#include "philox.cuh"

namespace mbis {
namespace {

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1) {
  const double u1 = ((double)a + 0.5) * 2.3283064365386963e-10;  // 2^-32
  const double u2 = ((double)b + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ double wrap_period(double x, double period) {
  double y = x - period * floor(x / period);
  if (y >= period) y -= period;
  if (y < 0.0) y += period;
  return y;
}

struct DrawConsts {
  double lpc[kMaxP];  // per-slot log-normalisation of the prior
};

__global__ void draw_kernel(DrawArgs a, DrawConsts k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint64_t g = (a.d_ctr0 ? *a.d_ctr0 : a.ctr0) + (uint64_t)i;
  double z[12];
#pragma unroll
  for (int blk = 0; blk < 3; ++blk) {
    if (4 * blk < a.P) {
      const Philox4 w = philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 2u, (uint32_t)blk, (uint32_t)a.seed,
                                      (uint32_t)(a.seed >> 32));
      box_muller(w.v[0], w.v[1], z[4 * blk], z[4 * blk + 1]);
      // the block's second pair only when a slot uses it (FP64 logarithms dominate the draw)
      if (4 * blk + 2 < a.P) box_muller(w.v[2], w.v[3], z[4 * blk + 2], z[4 * blk + 3]);
    }
  }
  double zz = 0.0;
  for (int p = 0; p < a.P; ++p) zz += z[p] * z[p];
  double lp = 0.0, mc = 0.0, q = 0.0;
  bool inside = true;
  for (int p = 0; p < a.P; ++p) {
    double x = a.mean[p];
    for (int r = 0; r <= p; ++r) x += a.scale * a.chol[p * kMaxP + r] * z[r];
    const int id = a.ids[p];
    if (id == kRa || id == kPhic) x = wrap_period(x, kTwoPi);
    if (id == kPsi) x = wrap_period(x, kPi);
    a.theta[(int64_t)p * a.n + i] = x;
    switch (id) {
      case kRa: case kPhic: case kPsi:
        lp += k.lpc[p];
        break;
      case kDec:
        inside = inside && x >= a.lo[p] && x <= a.hi[p];
        lp += log(cos(x)) + k.lpc[p];
        break;
      case kIota:
        inside = inside && x >= a.lo[p] && x <= a.hi[p];
        lp += log(sin(x)) + k.lpc[p];
        break;
      case kDl:
        inside = inside && x >= a.lo[p] && x <= a.hi[p];
        lp += 2.0 * log(x) + k.lpc[p];
        break;
      default:
        inside = inside && x >= a.lo[p] && x <= a.hi[p];
        lp += k.lpc[p];
        if (id == kMc) mc = x;
        if (id == kQ) q = x;
        break;
    }
  }
  if ((a.flags & MBIS_PRIOR_M1M2) && inside) {
    // |d(m1, m2)/d(Mc, q)| = Mc (1 + q)^(2/5) q^(-6/5) = [Mc^(5/2) (1 + q) / q^3]^(2/5): one
    // FP64 logarithm of a product instead of three
    lp += 0.4 * log(mc * mc * sqrt(mc) * (1.0 + q) / (q * q * q)) - a.log_mass_norm;
  }
  if (a.logp) a.logp[i] = inside ? lp : -INFINITY;
  if (a.logq) a.logq[i] = -0.5 * zz + a.log_q_const;
}

}  // namespace

cudaError_t launch_draw(const DrawArgs& a, cudaStream_t s) {
  DrawConsts k = {};
  for (int p = 0; p < a.P; ++p) {
    const int id = a.ids[p];
    const double lo = a.lo[p], hi = a.hi[p];
    switch (id) {
      case kRa: case kPhic: k.lpc[p] = -log(kTwoPi); break;
      case kPsi: k.lpc[p] = -log(kPi); break;
      case kDec: k.lpc[p] = -log(sin(hi) - sin(lo)); break;
      case kIota: k.lpc[p] = -log(cos(lo) - cos(hi)); break;
      case kDl: k.lpc[p] = log(3.0) - log(hi * hi * hi - lo * lo * lo); break;
      default:
        k.lpc[p] = ((a.flags & MBIS_PRIOR_M1M2) && (id == kMc || id == kQ)) ? 0.0 : -log(hi - lo);
        break;
    }
  }
  if (a.n <= 0) return cudaSuccess;
  const int threads = 128;
  const int64_t blocks = (a.n + threads - 1) / threads;
  draw_kernel<<<(unsigned)blocks, threads, 0, s>>>(a, k);
  return cudaGetLastError();
}

}  // namespace mbis
