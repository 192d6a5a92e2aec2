// k_loglike64.cu -- plain FP64 likelihood: the method of Eqs. 1-3 with the marginalised
// forms of Sec. III, every bin in double precision.  One warp per sample: lanes stride over
// frequency bins, a warp-shuffle reduction forms the overlaps, lane 0 applies the
// marginalisation.  This kernel is the double-precision GPU baseline that the mixed
// kernels are measured against, and the path of the FP64 workload.
//
// Per bin: Psi_k / 2pi = cst + sum_j C_j B_j(f_k) from the per-event basis table, the
// phasor e^(-i Psi_k) from sincospi, and the complex multiply-accumulate with the data
// table.  With fixed extrinsics the detectors are folded into one table; otherwise each
// detector adds its delay phase f_k dt_d and its own table.
//
// Time marginalisation: the per-bin integrand a_k = A sum_d P_d c_dk e^(-i phi_dk) of 32
// bins at a time is staged in shared memory; lane l accumulates
// Re z_j = sum_k Re(a_k) cos(2 pi f_k tau_j) + Im(a_k) sin(2 pi f_k tau_j) for the shifts
// j = l, l + 32, ...; the warp then takes ln mean_j exp(Re z_j - H/2).
#include "internal.h"
#include "marg.cuh"

namespace mbis {
namespace {

constexpr int kThreads64 = 256;
constexpr int kMaxShiftsPerLane = 8;  // up to 256 shifts

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct Response {
  double pr[kMaxDet], pim[kMaxDet], dt[kMaxDet];
};

// sum over detectors of c_dk e^(-i (Psi_k + 2 pi f_k dt_d)) weighted by P_d (the fold table
// already carries P_d and the delays)
__device__ __forceinline__ double2 bin_term(const LikeArgs& a, const PhaseCoeffs& pc, const Response& r, int32_t k) {
  const int32_t n = a.n_bins;
  double t = pc.cst;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) t = fma(pc.C[j], a.basis[(int64_t)j * n + k], t);
  if (a.fold) {
    double sn, cs;
    sincospi(2.0 * t, &sn, &cs);  // e^(-i Psi) = cs - i sn
    const double2 c = a.cfold64[k];
    return make_double2(c.x * cs + c.y * sn, c.y * cs - c.x * sn);
  }
  const double f = a.f_lo + (double)k * a.df;
  double zr = 0.0, zi = 0.0;
  for (int d = 0; d < a.n_det; ++d) {
    double sn, cs;
    sincospi(2.0 * fma(f, r.dt[d], t), &sn, &cs);
    const double2 c = a.cdet64[(int64_t)d * n + k];
    const double xr = c.x * cs + c.y * sn, xi = c.y * cs - c.x * sn;
    zr += r.pr[d] * xr - r.pim[d] * xi;
    zi += r.pr[d] * xi + r.pim[d] * xr;
  }
  return make_double2(zr, zi);
}

__global__ void __launch_bounds__(kThreads64) loglike_fp64_kernel(LikeArgs a) {
  __shared__ double2 sA[kThreads64 / 32][32];
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (s >= a.n) return;  // the whole warp leaves together

  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i) par[i] = a.pos[i] >= 0 ? a.theta[(int64_t)a.pos[i] * a.n + s] : a.fixed[i];
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

  Response r = {};
  double H = 0.0;
  if (a.fold) {
    H = A * A * a.tfold[kcut];
  } else {
    const double ci = cos(par[kIota]);
    for (int d = 0; d < a.n_det; ++d) {
      double fp, fc;
      antenna(a.det_x[d], a.det_y[d], par[kRa], par[kDec], par[kPsi], a.gmst, &fp, &fc);
      r.pr[d] = fp * 0.5 * (1.0 + ci * ci);
      r.pim[d] = -fc * ci;
      r.dt[d] = geocentre_delay(a.det_vertex[d], par[kRa], par[kDec], a.gmst);
      H += A * A * (r.pr[d] * r.pr[d] + r.pim[d] * r.pim[d]) * a.tdet[(int64_t)d * (n + 1) + kcut];
    }
  }

  if (a.marg == MBIS_MARG_TIME) {
    const int J = a.n_tshift;
    double zj[kMaxShiftsPerLane];
#pragma unroll
    for (int q = 0; q < kMaxShiftsPerLane; ++q) zj[q] = 0.0;
    for (int32_t k0 = 0; k0 < kcut; k0 += 32) {
      const int32_t k = k0 + lane;
      double2 t = make_double2(0.0, 0.0);
      if (k < kcut) {
        t = bin_term(a, pc, r, k);
        t.x *= A;
        t.y *= A;
      }
      sA[wib][lane] = t;
      __syncwarp();
      const int nk = min(32, kcut - k0);
      for (int kk = 0; kk < nk; ++kk) {
        const double2 ak = sA[wib][kk];
        const double2* tw = a.twiddle + (int64_t)(k0 + kk) * J;
#pragma unroll
        for (int q = 0; q < kMaxShiftsPerLane; ++q) {
          const int j = lane + 32 * q;
          if (j < J) {
            const double2 e = tw[j];
            zj[q] = fma(ak.x, e.x, fma(ak.y, e.y, zj[q]));
          }
        }
      }
      __syncwarp();
    }
    double m = -INFINITY;
#pragma unroll
    for (int q = 0; q < kMaxShiftsPerLane; ++q)
      if (lane + 32 * q < J) m = fmax(m, zj[q]);
    m = warp_max(m);
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxShiftsPerLane; ++q)
      if (lane + 32 * q < J) sum += exp(zj[q] - m);
    sum = warp_sum(sum);
    if (lane == 0) a.out[s] = m + log(sum / J) - 0.5 * H;
    return;
  }

  double zr = 0.0, zi = 0.0;
  for (int32_t k = lane; k < kcut; k += 32) {
    const double2 t = bin_term(a, pc, r, k);
    zr += t.x;
    zi += t.y;
  }
  zr = A * warp_sum(zr);
  zi = A * warp_sum(zi);
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
  const int64_t blocks = (a.n * 32 + kThreads64 - 1) / kThreads64;
  loglike_fp64_kernel<<<(unsigned)blocks, kThreads64, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mbis
