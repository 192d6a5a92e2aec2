// k_waveform.cu -- FP64 detector strains, Gaussian noise and inner products for the set-up
// helpers (synthetic injections, Fisher matrix).  Not on the per-sample path.
//   h_d(f) = (F+ h+(f) + Fx hx(f)) e^(-2 pi i f dt_d)                       (projection)
//   n_dk = sqrt(S_dk / (4 df)) (g1 + i g2), g from Philox (k, d, 1, 0)        (noise)
//   (a|b) = sum_d sum_k 4 df Re(conj(a_dk) b_dk) / S_dk                       (Eq. 1)
#include "internal.h"

namespace mbis {
namespace {

__device__ __forceinline__ void philox_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(m0, c[0]), lo0 = m0 * c[0];
    const uint32_t hi1 = __umulhi(m1, c[2]), lo1 = m1 * c[2];
    const uint32_t a = hi1 ^ c[1] ^ k0, b = hi0 ^ c[3] ^ k1;
    c[0] = a; c[1] = lo1; c[2] = b; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// grid: (bins, n_par); each thread one bin of one parameter vector, all detectors
__global__ void waveforms_kernel(int32_t n_par, const double* par_all, int32_t n_det, int32_t n_bins, double f_lo,
                                 double df, const double* geom, double gmst, double2* h_out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t m = blockIdx.y;
  if (k >= n_bins || m >= n_par) return;
  const double* par = par_all + (int64_t)m * kNumSlots;
  const double f = f_lo + (double)k * df;
  const bool live = k < live_bins(par[kMc], par[kQ], f_lo, df, n_bins);
  const PhaseCoeffs pc = phase_coeffs(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic]);
  double t = pc.cst;
  for (int j = 0; j < kNumBasis; ++j) t = fma(pc.C[j], basis(j, f), t);
  const double amp = live ? amplitude(par[kMc], par[kDl]) * pow(f, -7.0 / 6.0) : 0.0;
  const double ci = cos(par[kIota]);
  for (int d = 0; d < n_det; ++d) {
    const double* r = geom + 9 * d;
    double fp, fc;
    antenna(r + 3, r + 6, par[kRa], par[kDec], par[kPsi], gmst, &fp, &fc);
    const double dt = geocentre_delay(r, par[kRa], par[kDec], gmst);
    // P = F+ (1 + ci^2)/2 - i Fx ci ; h = amp P e^(-2 pi i (t + f dt))
    const double pr = fp * 0.5 * (1.0 + ci * ci), pi_ = -fc * ci;
    double sn, cs;
    sincospi(2.0 * fma(f, dt, t), &sn, &cs);
    const double er = cs, ei = -sn;
    h_out[((int64_t)m * n_det + d) * n_bins + k] = make_double2(amp * (pr * er - pi_ * ei), amp * (pr * ei + pi_ * er));
  }
}

__global__ void noise_kernel(int32_t n_det, int32_t n_bins, double df, const double* psd, uint64_t seed, double2* h) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t d = blockIdx.y;
  if (k >= n_bins || d >= n_det) return;
  uint32_t c[4] = {(uint32_t)k, (uint32_t)d, 1u, 0u};
  philox_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10, u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  const int64_t idx = (int64_t)d * n_bins + k;
  const double sig = sqrt(psd[idx] / (4.0 * df));
  double2 v = h[idx];
  v.x += sig * r * cs;
  v.y += sig * r * sn;
  h[idx] = v;
}

// one CTA per (a, b) pair
__global__ void inner_kernel(const double2* A, int32_t n_b, const double2* B, int32_t n_det, int32_t n_bins, double df,
                             const double* psd, double* out) {
  __shared__ double sh[256];
  const int32_t ia = blockIdx.x / n_b, ib = blockIdx.x % n_b;
  const int64_t len = (int64_t)n_det * n_bins;
  const double2* a = A + (int64_t)ia * len;
  const double2* b = B + (int64_t)ib * len;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) s += (a[i].x * b[i].x + a[i].y * b[i].y) / psd[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = 4.0 * df * sh[0];
}

}  // namespace

cudaError_t launch_waveforms(int32_t n_par, const double* par, int32_t n_det, int32_t n_bins, double f_lo, double df,
                             const DetResponse*, const double* det_geom, double gmst, double2* h_out, cudaStream_t s) {
  dim3 grid((n_bins + 255) / 256, n_par);
  waveforms_kernel<<<grid, 256, 0, s>>>(n_par, par, n_det, n_bins, f_lo, df, det_geom, gmst, h_out);
  return cudaGetLastError();
}

cudaError_t launch_noise(int32_t n_det, int32_t n_bins, double df, const double* psd, uint64_t seed, double2* h_io,
                         cudaStream_t s) {
  dim3 grid((n_bins + 255) / 256, n_det);
  noise_kernel<<<grid, 256, 0, s>>>(n_det, n_bins, df, psd, seed, h_io);
  return cudaGetLastError();
}

cudaError_t launch_inner_products(int32_t n_a, const double2* a, int32_t n_b, const double2* b, int32_t n_det,
                                  int32_t n_bins, double df, const double* psd, double* out, cudaStream_t s) {
  inner_kernel<<<n_a * n_b, 256, 0, s>>>(a, n_b, b, n_det, n_bins, df, psd, out);
  return cudaGetLastError();
}

}  // namespace mbis
