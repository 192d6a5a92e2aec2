// k_order.cu -- the order in which the likelihood kernels take the samples of a launch:
// most live bins first.  A CTA runs to the longest band among its samples (and a warp to the
// longest among its lanes), while a sample's result does not depend on which CTA or lanes
// it shares -- its bins past its own ISCO cut add exact zeros -- so ordering the samples by
// their live bins only removes the work a CTA would spend on its longest sample.
#include <algorithm>

#include "internal.h"

namespace mbis {
namespace {

// live bins of sample i in units of gran bins (rounded up), estimated in FP32: the estimate
// only steers the order; each CTA still runs to the exact cut of its samples
__device__ __forceinline__ int32_t order_key(const LikeArgs& a, int64_t i, int32_t gran) {
  const double mc = a.pos[kMc] >= 0 ? a.theta[(int64_t)a.pos[kMc] * a.n + i] : a.fixed[kMc];
  const double q = a.pos[kQ] >= 0 ? a.theta[(int64_t)a.pos[kQ] * a.n + i] : a.fixed[kQ];
  if (!(mc > 0.0) || !(q > 0.0)) return 0;
  const float qf = (float)q;
  const float m_sec = (float)(mc * kTsun) * powf(1.0f + qf, 1.2f) * powf(qf, -0.6f);
  const float fi = 1.0f / (46.172139f * m_sec);  // 6^(3/2) pi M
  const float k = fminf(fmaxf(ceilf((fi - (float)a.f_lo) / (float)a.df), 0.0f), (float)a.n_bins);
  return ((int32_t)k + gran - 1) / gran;
}

// warp-uniform loop over the samples; lanes with the same key add once per warp
__global__ void order_hist_kernel(LikeArgs a, int32_t gran, int32_t* hist) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int64_t i = base + lane;
    const bool on = i < a.n;
    const unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) {
      const int32_t key = order_key(a, i, gran);
      const unsigned peers = __match_any_sync(mask, key);
      if (lane == __ffs(peers) - 1) atomicAdd(&hist[key], __popc(peers));
    }
  }
}

// one CTA: counts -> first slot of each key, keys in decreasing order
__global__ void order_scan_kernel(int32_t n_keys, int32_t* hist) {
  __shared__ int32_t warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (n_keys + (int)blockDim.x - 1) / (int)blockDim.x;
  const int r0 = t * per, r1 = min(r0 + per, n_keys);  // ranks r: key n_keys - 1 - r
  int32_t local = 0;
  for (int r = r0; r < r1; ++r) local += hist[n_keys - 1 - r];
  int32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)blockDim.x >> 5;
    int32_t v = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) warp_tot[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  int32_t run = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0);
  for (int r = r0; r < r1; ++r) {
    const int32_t c = hist[n_keys - 1 - r];
    hist[n_keys - 1 - r] = run;
    run += c;
  }
}

__global__ void order_scatter_kernel(LikeArgs a, int32_t gran, int32_t* next, int32_t* perm) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int64_t i = base + lane;
    const bool on = i < a.n;
    const unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) {
      const int32_t key = order_key(a, i, gran);
      const unsigned peers = __match_any_sync(mask, key);
      const int leader = __ffs(peers) - 1;
      int32_t first = 0;
      if (lane == leader) first = atomicAdd(&next[key], __popc(peers));
      first = __shfl_sync(peers, first, leader);
      perm[first + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

}  // namespace

int32_t order_keys(int32_t n_bins, int32_t gran) { return (n_bins + gran - 1) / gran + 1; }

cudaError_t launch_sample_order(const LikeArgs& a, int32_t gran, int32_t* hist, int32_t* perm, cudaStream_t s) {
  const int32_t n_keys = order_keys(a.n_bins, gran);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)n_keys, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>((a.n + 255) / 256, 4 * 152);
  order_hist_kernel<<<grid, 256, 0, s>>>(a, gran, hist);
  order_scan_kernel<<<1, 1024, 0, s>>>(n_keys, hist);
  order_scatter_kernel<<<grid, 256, 0, s>>>(a, gran, hist, perm);
  return cudaGetLastError();
}

}  // namespace mbis
