// k_levels.cu -- credible level of a reference point under importance weights, the quantity
// of the P-P self-consistency test (Sec. III A): for each sampled slot, the weighted fraction
// of the samples below the reference, ties counting half.  One CTA per slot strides over
// the samples and reduces in a fixed order (FP64, deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace mbis {
namespace {

constexpr int kLevelThreads = 512;
constexpr int kMaxLevelSlots = 16;

struct LevelRef {
  double r[kMaxLevelSlots];
};

__global__ void __launch_bounds__(kLevelThreads) levels_kernel(int64_t n, const double* __restrict__ theta,
                                                               const double* __restrict__ w, LevelRef ref,
                                                               double* __restrict__ out) {
  __shared__ double s_below[kLevelThreads], s_tot[kLevelThreads];
  const int p = blockIdx.x;
  const double r = ref.r[p];
  const double* x = theta + (int64_t)p * n;
  double below = 0.0, tot = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kLevelThreads) {
    const double wi = w[i];
    if (!(wi > 0.0)) continue;
    const double xi = x[i];
    tot += wi;
    below += xi < r ? wi : (xi == r ? 0.5 * wi : 0.0);
  }
  s_below[threadIdx.x] = below;
  s_tot[threadIdx.x] = tot;
  __syncthreads();
  for (int o = kLevelThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_below[threadIdx.x] += s_below[threadIdx.x + o];
      s_tot[threadIdx.x] += s_tot[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = s_tot[0] > 0.0 ? s_below[0] / s_tot[0] : NAN;
}

}  // namespace
}  // namespace mbis

extern "C" mbis_status mbis_credible_levels(int64_t n, int32_t P, const double* theta, const double* weights,
                                            const double* ref, double* levels, void* stream) {
  if (n < 1 || P < 1 || P > mbis::kMaxLevelSlots || !theta || !weights || !ref || !levels) {
    mbis::set_last_error("mbis_credible_levels: need n >= 1, 1 <= P <= 16 and non-null buffers");
    return MBIS_E_INVALID;
  }
  mbis::LevelRef r = {};
  for (int p = 0; p < P; ++p) r.r[p] = ref[p];
  mbis::levels_kernel<<<P, mbis::kLevelThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, theta, weights, r, levels);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mbis::set_last_error(std::string("mbis_credible_levels: ") + cudaGetErrorString(e));
    return MBIS_E_CUDA;
  }
  return MBIS_OK;
}
