// k_reduce.cu -- importance weights (Eq. 5), Kish ESS (Eq. 6) and evidence, in two passes.
//   pass 1: m = max_i (log L_i + log pi_i - log g_i)
//   pass 2: S1 = sum e^(log w_i - m), S2 = sum e^(2 (log w_i - m))   (FP64)
//   pass 3 (optional): w_i = e^(log w_i - m) / S1
// Each pass runs a fixed grid (4 CTAs per SM); per-CTA partials go to device scratch and
// the last CTA to finish (atomic ticket) folds them in a fixed order, so the result does
// not depend on scheduling.  The ticket counter returns to zero at the end of each pass.
#include "internal.h"

namespace mbis {
namespace {

__device__ __forceinline__ double log_weight(const double* ll, const double* lp, const double* lq, int64_t i) {
  return ll[i] + lp[i] - lq[i];
}

template <int OP>  // 0: max, 1: sum
__device__ __forceinline__ double block_fold(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = OP == 0 ? fmax(sh[t], sh[t + s]) : sh[t] + sh[t + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

__global__ void __launch_bounds__(kReduceThreads) reduce_max_kernel(int64_t n, const double* ll, const double* lp,
                                                                    const double* lq, ReduceScratch scr) {
  __shared__ double sh[kReduceThreads];
  double m = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double lw = log_weight(ll, lp, lq, i);
    if (lw > m) m = lw;
  }
  m = block_fold<0>(m, sh);
  if (threadIdx.x == 0) scr.partials[blockIdx.x] = m;
  if (last_block(scr.counter)) {
    double v = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v = fmax(v, ((volatile double*)scr.partials)[b]);
    v = block_fold<0>(v, sh);
    if (threadIdx.x == 0) {
      scr.result[0] = v;
      scr.result[3] = (double)n;
      *scr.counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(kReduceThreads) reduce_sum_kernel(int64_t n, const double* ll, const double* lp,
                                                                    const double* lq, ReduceScratch scr) {
  __shared__ double sh[kReduceThreads];
  const double m = scr.result[0];
  double s1 = 0.0, s2 = 0.0;
  if (m > -INFINITY) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const double e = exp(log_weight(ll, lp, lq, i) - m);
      s1 += e;
      s2 += e * e;
    }
  }
  s1 = block_fold<1>(s1, sh);
  s2 = block_fold<1>(s2, sh);
  if (threadIdx.x == 0) {
    scr.partials[2 * blockIdx.x] = s1;
    scr.partials[2 * blockIdx.x + 1] = s2;
  }
  if (last_block(scr.counter)) {
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      volatile double* p = scr.partials;
      for (int k = 0; k < (int)gridDim.x; ++k) {
        a += p[2 * k];
        b += p[2 * k + 1];
      }
      scr.result[1] = a;
      scr.result[2] = b;
      *scr.counter = 0u;
    }
  }
}

__global__ void weights_kernel(int64_t n, const double* ll, const double* lp, const double* lq, const double* result,
                               double* w) {
  const double m = result[0], inv = 1.0 / result[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = m > -INFINITY ? exp(log_weight(ll, lp, lq, i) - m) * inv : 0.0;
}

}  // namespace

cudaError_t launch_reduce(int64_t n, const double* loglike, const double* logp, const double* logq, double* weights,
                          const ReduceScratch& scr, cudaStream_t s) {
  reduce_max_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, loglike, logp, logq, scr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_sum_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, loglike, logp, logq, scr);
  e = cudaGetLastError();
  if (e != cudaSuccess || weights == nullptr) return e;
  weights_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, loglike, logp, logq, scr.result, weights);
  return cudaGetLastError();
}

}  // namespace mbis
