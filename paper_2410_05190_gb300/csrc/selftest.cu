// selftest.cu -- exercises the bounded device-side wait that every kernel of the library
// uses on its mbarriers (a wait on a barrier that nothing completes must give up after its
// limit and report MBIS_E_TIMEOUT, leaving the CUDA context usable), and exposes the
// float-float sine and cosine of the time-marginalised kernel's set-up for an accuracy test.
#include "internal.h"
#include "ffloat.cuh"
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

}  // namespace

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
