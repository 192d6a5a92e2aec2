// selftest.cu -- exercises the bounded device-side wait that every kernel of the library
// uses on its mbarriers (a wait on a barrier that nothing completes must give up after its
// limit and report MBIS_E_TIMEOUT, leaving the CUDA context usable), and exposes the
// float-float sine and cosine and per-sample set-up of the time-marginalised kernel for
// accuracy tests against their FP64 counterparts.
#include "internal.h"
#include "ffloat.cuh"
#include "setup_ff.cuh"
#include "tc.cuh"

namespace {

__global__ void wait_never_kernel(uint64_t limit_ns, int32_t* status, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbis::tc::mbar_init(&bar, 1);  // expects one arrival that never comes
    mbis::tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = mbis::tc::global_ns();
    const bool ok = mbis::tc::mbar_wait(&bar, 0u, limit_ns);
    *waited_ns = mbis::tc::global_ns() - t0;
    *status = ok ? (int32_t)MBIS_OK : (int32_t)MBIS_E_TIMEOUT;
  }
}

__global__ void ff_sincos_kernel(int64_t n, const double* __restrict__ x, double* s, double* c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sv, cv;
  mbis::ff_sincos_d(x[i], sv, cv);
  if (s) s[i] = sv;
  if (c) c[i] = cv;
}

// out: [2][12][n] -- row block 0 the FP64 sample_setup, row block 1 the float-float one:
// C_0..C_8, cst, amp, kcut (as a double)
__global__ void setup_pair_kernel(int64_t n, const double* __restrict__ p, double f_lo, double df, int32_t n_bins,
                                  double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) v[k] = p[k * n + i];
  const mbis::SampleSetup a = mbis::sample_setup(v[0], v[1], v[2], v[3], v[4], v[5], v[6], f_lo, df, n_bins);
  const mbis::SampleSetupFF b = mbis::sample_setup_ff(v[0], v[1], v[2], v[3], v[4], v[5], v[6], f_lo, df, n_bins);
  for (int j = 0; j < mbis::kNumBasis; ++j) {
    out[j * n + i] = a.pc.C[j];
    out[(12 + j) * n + i] = mbis::ff_to_double(b.C[j]);
  }
  out[9 * n + i] = a.pc.cst;
  out[21 * n + i] = mbis::ff_to_double(b.cst);
  out[10 * n + i] = a.amp;
  out[22 * n + i] = b.amp;
  out[11 * n + i] = (double)a.kcut;
  out[23 * n + i] = (double)b.kcut;
}

}  // namespace

extern "C" mbis_status mbis_debug_setup_pair(int64_t n, const double* params, double f_lo, double df, int32_t n_bins,
                                             double* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!params || !out)) || !(df > 0.0) || n_bins < 1) {
    mbis::set_last_error("mbis_debug_setup_pair: need n >= 0, non-null buffers, df > 0, n_bins >= 1");
    return MBIS_E_INVALID;
  }
  if (n == 0) return MBIS_OK;
  setup_pair_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)cuda_stream>>>(n, params, f_lo, df, n_bins,
                                                                                       out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mbis::set_last_error(std::string("mbis_debug_setup_pair: ") + cudaGetErrorString(e));
    return MBIS_E_CUDA;
  }
  return MBIS_OK;
}

extern "C" mbis_status mbis_debug_ff_sincos(int64_t n, const double* x, double* sin_out, double* cos_out,
                                            void* cuda_stream) {
  if (n < 0 || (n > 0 && !x)) {
    mbis::set_last_error("mbis_debug_ff_sincos: need n >= 0 and x non-null");
    return MBIS_E_INVALID;
  }
  if (n == 0) return MBIS_OK;
  ff_sincos_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(n, x, sin_out, cos_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mbis::set_last_error(std::string("mbis_debug_ff_sincos: ") + cudaGetErrorString(e));
    return MBIS_E_CUDA;
  }
  return MBIS_OK;
}

extern "C" mbis_status mbis_debug_wait_timeout(uint64_t limit_ns, int32_t* status_out, uint64_t* waited_ns_out) {
  if (!status_out || limit_ns == 0 || limit_ns > 2000000000ull) {
    mbis::set_last_error("mbis_debug_wait_timeout: status_out must be non-null, 0 < limit_ns <= 2e9");
    return MBIS_E_INVALID;
  }
  int32_t* d_status = nullptr;
  unsigned long long* d_ns = nullptr;
  cudaError_t e = cudaMalloc(&d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_ns, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    wait_never_kernel<<<1, 32>>>(limit_ns, d_status, d_ns);
    e = cudaGetLastError();
  }
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpy(status_out, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
  if (d_status) cudaFree(d_status);
  if (d_ns) cudaFree(d_ns);
  if (e != cudaSuccess) {
    mbis::set_last_error(std::string("mbis_debug_wait_timeout: ") + cudaGetErrorString(e));
    return MBIS_E_CUDA;
  }
  if (waited_ns_out) *waited_ns_out = ns;
  return MBIS_OK;
}
