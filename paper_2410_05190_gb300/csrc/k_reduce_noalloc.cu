// k_reduce_noalloc.cu -- the weight reduction (importance weights, ESS, evidence) for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc once it is running -- a low-latency
// serving loop in which an allocation would synchronise the device and stall other work,
// or a host framework that owns all device memory and forbids allocations after start-up.
// mbis_reduce keeps its scratch in the context, which mbis_create allocates; this variant
// needs no context and keeps its scratch in the fixed array below instead.
//
// The array lives for as long as the library is loaded, on every GPU that loads it
// (about 128 KiB each).  With lazy module loading (the CUDA default) the module that holds
// it is placed on a device by the first call there: a one-time device allocation, which
// callers avoid on their critical path by calling once at start-up (e.g. with n = 1).  It holds per-CTA partial results for at most kMaxPartials CTAs of
// kItems samples, so one call handles at most kMaxSamples = 2^24 samples; larger requests
// are rejected.  Every call shares the one array and it keeps the last call's contents:
// each call clears the ticket counter it relies on before launching, and calls whose work
// overlaps on the GPU (different streams, or host threads) race on the array -- serialise
// them on one stream.
#include <mutex>

#include "internal.h"

namespace mbis {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int64_t kItems = (int64_t)kThreads * kPerThread;  // samples per CTA
constexpr int kMaxPartials = 8192;                           // CTAs per call
constexpr int64_t kMaxSamples = kItems * kMaxPartials;       // 2^24
constexpr int kResult = 2 * kMaxPartials;                    // result slots: m, s1, s2, n
constexpr int kCounter = kResult + 4;                        // ticket counter (as uint32)
constexpr int kMaxDevices = 64;

// partials [2 * kMaxPartials] | result [4] | counter [1] | pad
static __device__ __align__(256) double g_reduce_scratch[kResult + 8];

// device address of the array per device, filled on the first successful lookup
std::mutex g_scratch_mu;
double* g_scratch[kMaxDevices] = {};

__device__ __forceinline__ double lw_at(const double* ll, const double* lp, const double* lq, int64_t i) {
  return ll[i] + lp[i] - lq[i];
}

__device__ __forceinline__ double cta_fold(double v, double* sh, bool take_max) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = take_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + s]) : sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool is_last_cta(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

__global__ void __launch_bounds__(kThreads) noalloc_max_kernel(int64_t n, const double* ll, const double* lp,
                                                               const double* lq, double* scratch) {
  __shared__ double sh[kThreads];
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounter);
  const int64_t base = (int64_t)blockIdx.x * kItems;
  double m = -INFINITY;
#pragma unroll
  for (int r = 0; r < kPerThread; ++r) {
    const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
    if (i < n) m = fmax(m, lw_at(ll, lp, lq, i));
  }
  m = cta_fold(m, sh, true);
  if (threadIdx.x == 0) scratch[blockIdx.x] = m;
  if (is_last_cta(counter)) {
    double v = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) v = fmax(v, ((volatile double*)scratch)[b]);
    v = cta_fold(v, sh, true);
    if (threadIdx.x == 0) {
      scratch[kResult] = v;
      scratch[kResult + 3] = (double)n;
      *counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_sum_kernel(int64_t n, const double* ll, const double* lp,
                                                               const double* lq, double* scratch) {
  __shared__ double sh[kThreads];
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounter);
  const double m = scratch[kResult];
  const int64_t base = (int64_t)blockIdx.x * kItems;
  double s1 = 0.0, s2 = 0.0;
  if (m > -INFINITY) {
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
      if (i < n) {
        const double e = exp(lw_at(ll, lp, lq, i) - m);
        s1 += e;
        s2 += e * e;
      }
    }
  }
  s1 = cta_fold(s1, sh, false);
  s2 = cta_fold(s2, sh, false);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = s1;
    scratch[2 * blockIdx.x + 1] = s2;
  }
  if (is_last_cta(counter) && threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    volatile double* p = scratch;
    for (int k = 0; k < (int)gridDim.x; ++k) {
      a += p[2 * k];
      b += p[2 * k + 1];
    }
    scratch[kResult + 1] = a;
    scratch[kResult + 2] = b;
    *counter = 0u;
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_weights_kernel(int64_t n, const double* ll, const double* lp,
                                                                   const double* lq, const double* scratch,
                                                                   double* w) {
  const double m = scratch[kResult], inv = 1.0 / scratch[kResult + 1];
  const int64_t base = (int64_t)blockIdx.x * kItems;
#pragma unroll
  for (int r = 0; r < kPerThread; ++r) {
    const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
    if (i < n) w[i] = m > -INFINITY ? exp(lw_at(ll, lp, lq, i) - m) * inv : 0.0;
  }
}

// With the device current: the device address of the scratch array, looked up on the first
// call that succeeds on that device and kept.  A failed lookup (e.g. one made during a
// stream capture) is not kept: the next call tries again.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();  // reported here; keep it out of the next call's launch check
      return e;
    }
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

void fill_summary(const double* r, int64_t n, mbis_summary* out) {
  const double m = r[0], s1 = r[1], s2 = r[2];
  out->max_logw = m;
  out->s1 = s1;
  out->s2 = s2;
  out->n = n;
  out->all_zero = !(m > -INFINITY) || !(s1 > 0.0);
  out->ess = s2 > 0.0 ? s1 * s1 / s2 : 0.0;
  out->log_z = (m > -INFINITY && s1 > 0.0 && n > 0) ? m + log(s1) - log((double)n) : -INFINITY;
}

}  // namespace
}  // namespace mbis

extern "C" mbis_status mbis_reduce_noalloc(int64_t n, const double* loglike, const double* log_prior,
                                           const double* log_q, double* weights_out, mbis_summary* out,
                                           void* cuda_stream) {
  using namespace mbis;
  if (!out || n < 0 || (n > 0 && (!loglike || !log_prior || !log_q))) {
    set_last_error("mbis_reduce_noalloc: null buffer or negative n");
    return MBIS_E_INVALID;
  }
  if (n > kMaxSamples) {
    set_last_error("mbis_reduce_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                   std::to_string(kMaxSamples) + " samples per call (use mbis_reduce, or split the batch)");
    return MBIS_E_INVALID;
  }
  if (n == 0) {
    const double r[3] = {-INFINITY, 0.0, 0.0};
    fill_summary(r, 0, out);
    return MBIS_OK;
  }
  auto cuda_fail = [](const char* what, cudaError_t e) {
    set_last_error(std::string("mbis_reduce_noalloc: ") + what + ": " + cudaGetErrorString(e));
    return MBIS_E_CUDA;
  };
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress", e);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const unsigned grid = (unsigned)((n + kItems - 1) / kItems);
  // the ticket counter must start at zero whatever an earlier call left behind
  if ((e = cudaMemsetAsync(scratch + kCounter, 0, sizeof(unsigned int), s)) != cudaSuccess)
    return cuda_fail("cudaMemsetAsync", e);
  noalloc_max_kernel<<<grid, kThreads, 0, s>>>(n, loglike, log_prior, log_q, scratch);
  noalloc_sum_kernel<<<grid, kThreads, 0, s>>>(n, loglike, log_prior, log_q, scratch);
  if (weights_out) noalloc_weights_kernel<<<grid, kThreads, 0, s>>>(n, loglike, log_prior, log_q, scratch, weights_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("launch", e);
  double r[3];
  if ((e = cudaMemcpyAsync(r, scratch + kResult, sizeof(r), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail("cudaMemcpyAsync", e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
  fill_summary(r, n, out);
  return MBIS_OK;
}
