// k_moments.cu -- weighted mean and covariance of the proposal samples, for refitting the
// Gaussian proposal from an importance-weighted batch (the iterative update of the proposal
// that Sec. III A suggests).
//
// With normalised weights w_i and offsets d_i = theta_i - ref (periodic slots wrapped into
// [-period/2, period/2) around ref), the kernel accumulates sum w d and sum w d d^T in FP64;
// offsets keep the sums well conditioned for parameters measured to ~1e-5 relative.
// Fixed grid, per-CTA partials in device scratch, last CTA folds them in a fixed order.
#include "internal.h"

namespace mbis {
namespace {

constexpr int kMomThreads = 128;
constexpr int kMomBlocks = 304;  // 2 per SM

__global__ void __launch_bounds__(kMomThreads) moments_kernel(int64_t n, int32_t P, const double* theta,
                                                              const double* w, MomentArgs ma, double* partials,
                                                              unsigned int* counter, double* out) {
  const int nm = 1 + P + P * (P + 1) / 2;  // sum of weights, first moments, upper triangle
  double acc[1 + kMaxP + kMaxP * (kMaxP + 1) / 2];
  for (int m = 0; m < nm; ++m) acc[m] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    if (!(wi > 0.0)) continue;
    double d[kMaxP];
    for (int p = 0; p < P; ++p) {
      double x = theta[(int64_t)p * n + i] - ma.ref[p];
      const double T = ma.period[p];
      if (T > 0.0) x -= T * floor(x / T + 0.5);
      d[p] = x;
    }
    int m = 0;
    acc[m++] += wi;
    for (int p = 0; p < P; ++p) acc[m++] += wi * d[p];
    for (int p = 0; p < P; ++p)
      for (int q = p; q < P; ++q) acc[m++] += wi * d[p] * d[q];
  }
  __shared__ double sh[kMomThreads];
  __shared__ bool last;
  for (int m = 0; m < nm; ++m) {
    sh[threadIdx.x] = acc[m];
    __syncthreads();
    for (int s = kMomThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * nm + m] = sh[0];
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    for (int m = threadIdx.x; m < nm; m += blockDim.x) {
      double s = 0.0;
      volatile double* p = partials;
      for (int b = 0; b < (int)gridDim.x; ++b) s += p[(int64_t)b * nm + m];
      out[m] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

}  // namespace

int moments_partials_size(int32_t P) { return kMomBlocks * (1 + P + P * (P + 1) / 2); }

cudaError_t launch_moments(int64_t n, int32_t P, const double* theta, const double* w, const MomentArgs& ma,
                           double* partials, unsigned int* counter, double* out, cudaStream_t s) {
  moments_kernel<<<kMomBlocks, kMomThreads, 0, s>>>(n, P, theta, w, ma, partials, counter, out);
  return cudaGetLastError();
}

}  // namespace mbis
