// k_loglike64.cu -- plain FP64 likelihood: the method of Eqs. 1-3 with the marginalised
// forms of Sec. III, every bin in double precision.  One warp per sample: lanes stride over
// frequency bins, a warp-shuffle reduction forms the overlaps, lane 0 applies the
// marginalisation.  This kernel is the double-precision GPU baseline that the mixed kernel
// is measured against, and the path of the FP64 workload.
//
// Per bin: Psi_k / 2pi = cst + sum_j C_j B_j(f_k) from the per-event basis table, the
// phasor e^(-i Psi_k) from sincospi, and the complex multiply-accumulate with the data
// table.  With fixed extrinsics the detectors are folded into one table; otherwise each
// detector adds its delay phase f_k dt_d and its own table.
#include "internal.h"
#include "marg.cuh"

namespace mbis {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) loglike_fp64_kernel(LikeArgs a) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= a.n) return;  // the whole warp leaves together

  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i) par[i] = a.fixed[i];
  for (int p = 0; p < a.P; ++p) par[a.ids[p]] = a.theta[(int64_t)p * a.n + s];
  if (a.marg & MBIS_MARG_PHASE) par[kPhic] = 0.0;
  if (a.marg & MBIS_MARG_DISTANCE) par[kDl] = 1.0;
  const bool valid = par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 && fabs(par[kChi2]) < 1.0 &&
                     par[kDl] > 0.0 && isfinite(par[kTc]) && isfinite(par[kPhic]) && isfinite(par[kRa]) &&
                     isfinite(par[kDec]) && isfinite(par[kPsi]) && isfinite(par[kIota]);
  if (!valid) {
    if (lane == 0) a.out[s] = -INFINITY;
    return;
  }
  const PhaseCoeffs pc = phase_coeffs(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic]);
  const int32_t kcut = live_bins(par[kMc], par[kQ], a.f_lo, a.df, a.n_bins);
  const double A = amplitude(par[kMc], par[kDl]);
  const int32_t n = a.n_bins;

  double zr = 0.0, zi = 0.0, H = 0.0;
  if (a.fold) {
    for (int32_t k = lane; k < kcut; k += 32) {
      double t = pc.cst;
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) t = fma(pc.C[j], a.basis[(int64_t)j * n + k], t);
      double sn, cs;
      sincospi(2.0 * t, &sn, &cs);  // e^(-i Psi) = cs - i sn
      const double2 c = a.cfold64[k];
      zr += c.x * cs + c.y * sn;
      zi += c.y * cs - c.x * sn;
    }
    zr = warp_sum(zr);
    zi = warp_sum(zi);
    H = A * A * a.tfold[kcut];
    zr *= A;
    zi *= A;
  } else {
    double pr[kMaxDet], pim[kMaxDet], dt[kMaxDet], zdr[kMaxDet], zdi[kMaxDet];
    const double ci = cos(par[kIota]);
    for (int d = 0; d < a.n_det; ++d) {
      double fp, fc;
      antenna(a.det_x[d], a.det_y[d], par[kRa], par[kDec], par[kPsi], a.gmst, &fp, &fc);
      pr[d] = fp * 0.5 * (1.0 + ci * ci);
      pim[d] = -fc * ci;
      dt[d] = geocentre_delay(a.det_vertex[d], par[kRa], par[kDec], a.gmst);
      zdr[d] = 0.0;
      zdi[d] = 0.0;
    }
    for (int32_t k = lane; k < kcut; k += 32) {
      double t = pc.cst;
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) t = fma(pc.C[j], a.basis[(int64_t)j * n + k], t);
      const double f = a.f_lo + (double)k * a.df;
      for (int d = 0; d < a.n_det; ++d) {
        double sn, cs;
        sincospi(2.0 * fma(f, dt[d], t), &sn, &cs);
        const double2 c = a.cdet64[(int64_t)d * n + k];
        zdr[d] += c.x * cs + c.y * sn;
        zdi[d] += c.y * cs - c.x * sn;
      }
    }
    for (int d = 0; d < a.n_det; ++d) {
      const double r = warp_sum(zdr[d]), im = warp_sum(zdi[d]);
      zr += A * (pr[d] * r - pim[d] * im);
      zi += A * (pr[d] * im + pim[d] * r);
      H += A * A * (pr[d] * pr[d] + pim[d] * pim[d]) * a.tdet[(int64_t)d * (n + 1) + kcut];
    }
  }
  if (lane != 0) return;
  double ll;
  if (a.marg == 0) {
    ll = zr - 0.5 * H;
  } else if (a.marg == MBIS_MARG_PHASE) {
    ll = log_i0(hypot(zr, zi)) - 0.5 * H;
  } else {  // PHASE | DISTANCE
    ll = log_distance_marginal(hypot(zr, zi), H, a.dmin, a.dmax, a.gl);
  }
  a.out[s] = ll;
}

}  // namespace

cudaError_t launch_loglike_fp64(const LikeArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (a.n * 32 + threads - 1) / threads;
  loglike_fp64_kernel<<<(unsigned)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mbis
