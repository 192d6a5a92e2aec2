// k_rb.cu -- relative binning (the heterodyned likelihood of Zackay, Dai & Venumadhav 2018;
// the paper notes that faster likelihoods such as this plug into its method, Sec. IV) for
// contexts whose extrinsic parameters are fixed, so that the detectors fold into one table.
//
// About a fiducial theta0 the template's ratio to the fiducial, r(f) = (A / A0)
// e^(-i 2 pi (Psi(f) - Psi0(f))), is smooth; inside each coarse bin [f_b, f_b+1) it is
// replaced by its chord through the bin's edges.  With the fiducial-heterodyned data weights
// W_k = c_k e^(-i 2 pi Psi0(f_k)) (c the folded data table, which carries the detector
// responses, delays, f^(-7/6), 1/S and 4 df), the overlap becomes
//   Z = A sum_b [rho(f_b) A0_b + (rho(f_b+1) - rho(f_b)) / (f_b+1 - f_b) A1_b],
//   A0_b = sum_{k in b} W_k,  A1_b = sum_{k in b} W_k (f_k - f_b),  rho = e^(-i 2 pi dPsi),
// the bin holding the sample's ISCO cut summed only below it (from prefix sums); <h|h> stays
// exact (the amplitude prefix table).  Per sample the phase is evaluated at the n_rb + 1
// edges only: its difference from the fiducial's, in FP32 from FP64 coefficient
// differences, then MUFU sine / cosine; the chord sums run in FP32 over chunks of 16 bins
// whose sums are gathered as float pairs (no FP64 arithmetic in the loop over bins).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ffloat.cuh"
#include "internal.h"
#include "marg.cuh"

namespace mbis {
namespace {

constexpr int kRbThreads = 512;
constexpr int kRbChunk = 16;
constexpr size_t kRbSmemMax = 112 * 1024;  // records staged in shared memory up to 1791 bins
constexpr float kTwoPiF = 6.28318530717958647692f;

// W_k and (f_k - f_lo) W_k as four real rows [re W, im W, re fW, im fW][n]
__global__ void rb_weights_kernel(int32_t n, const double2* __restrict__ c, const double* __restrict__ basis,
                                  PhaseCoeffs pc0, double f_lo, double df, double* out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double t = pc0.cst;
  for (int j = 0; j < kNumBasis; ++j) t = fma(pc0.C[j], basis[(int64_t)j * n + k], t);
  t -= floor(t);
  double s, co;
  sincospi(2.0 * t, &s, &co);  // e^(-i 2 pi t) = co - i s
  const double2 ck = c[k];
  const double wr = ck.x * co + ck.y * s, wi = ck.y * co - ck.x * s;
  const double fk = (double)k * df;
  out[k] = wr;
  out[(int64_t)n + k] = wi;
  out[2 * (int64_t)n + k] = fk * wr;
  out[3 * (int64_t)n + k] = fk * wi;
}

// One coarse-bin record (64 bytes): basis_j at the bin's left edge, 1 / width, the edge's bin
// index, and the bin's sums (A0, A1) / scale; record n_rb carries the last edge only.
struct RbRec {
  float be[kNumBasis];
  float invw;
  int32_t k0;
  float pad;
  float4 sum;
};
static_assert(sizeof(RbRec) == 64, "coarse-bin record is 64 bytes");

__global__ void rb_summary_kernel(int32_t n_rb, int32_t n, const int32_t* __restrict__ edges,
                                  const double* __restrict__ T, double f_lo, double df, double inv_scale,
                                  RbRec* rec) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > n_rb) return;
  RbRec r = {};
  const double fe = f_lo + (double)edges[b] * df;
  for (int j = 0; j < kNumBasis; ++j) r.be[j] = (float)basis(j, fe);
  r.k0 = edges[b];
  if (b < n_rb) {
    const int32_t k0 = edges[b], k1 = edges[b + 1];
    const int64_t m = (int64_t)n + 1;
    const double a0r = T[k1] - T[k0], a0i = T[m + k1] - T[m + k0];
    const double ofs = (double)k0 * df;  // f_b - f_lo
    const double a1r = (T[2 * m + k1] - T[2 * m + k0]) - ofs * a0r;
    const double a1i = (T[3 * m + k1] - T[3 * m + k0]) - ofs * a0i;
    r.sum = make_float4((float)(a0r * inv_scale), (float)(a0i * inv_scale), (float)(a1r * inv_scale),
                        (float)(a1i * inv_scale));
    r.invw = (float)(1.0 / ((double)(k1 - k0) * df));
  }
  rec[b] = r;
}

struct RbArgs {
  LikeArgs la;
  int32_t n_rb;
  const RbRec* rec;      // [n_rb + 1]
  int32_t rec_smem;      // stage the records in shared memory
  const double* prefix;  // [4][n_bins + 1]
  double scale;
  double C0[kNumBasis], cst0;
};

__device__ __forceinline__ float2 rho_at(const RbRec& r, const float* dC, float dcst) {
  float t = dcst;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) t = fmaf(dC[j], r.be[j], t);
  t -= rintf(t);  // turns in [-1/2, 1/2]
  float s, c;
  __sincosf(-kTwoPiF * t, &s, &c);
  return make_float2(c, s);  // e^(-i 2 pi t)
}

__device__ __forceinline__ void cmac(float2 a, float2 b, float& zr, float& zi) {
  zr = fmaf(a.x, b.x, fmaf(-a.y, b.y, zr));
  zi = fmaf(a.x, b.y, fmaf(a.y, b.x, zi));
}

__global__ void __launch_bounds__(kRbThreads, 2) rb_loglike_kernel(RbArgs r) {
  extern __shared__ RbRec s_rec[];
  const LikeArgs& a = r.la;
  const RbRec* recs = r.rec;
  if (r.rec_smem) {
    const float4* src = reinterpret_cast<const float4*>(r.rec);
    float4* dst = reinterpret_cast<float4*>(s_rec);
    for (int i = threadIdx.x; i < 4 * (r.n_rb + 1); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    recs = s_rec;
  }
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i) par[i] = a.pos[i] >= 0 ? a.theta[(int64_t)a.pos[i] * a.n + s] : a.fixed[i];
  const bool valid = par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 && fabs(par[kChi2]) < 1.0 &&
                     ((a.marg & MBIS_MARG_DISTANCE) || par[kDl] > 0.0) && isfinite(par[kTc]) && isfinite(par[kPhic]);
  if (!valid) {
    a.out[s] = -INFINITY;
    return;
  }
  const double dl = (a.marg & MBIS_MARG_DISTANCE) ? 1.0 : par[kDl];
  const MassSetup ms = mass_setup(par[kMc], par[kQ], dl);
  const PhaseCoeffs pc = phase_coeffs_a(par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic], ms.a, ms.la, ms.a13);
  const int32_t kcut = live_bins_m(ms.m_sec, a.f_lo, a.df, a.n_bins);
  float dC[kNumBasis];
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) dC[j] = (float)(pc.C[j] - r.C0[j]);
  const float dcst = (float)(pc.cst - r.cst0);

  FFSum zr_all, zi_all;        // the chunk sums (scaled), added without FP64 arithmetic
  double zr64 = 0.0, zi64 = 0.0;  // the partial bin at the ISCO cut (FP64 prefix sums)
  float zr = 0.f, zi = 0.f;
  RbRec cur = recs[0];
  float2 rho = rho_at(cur, dC, dcst);
  for (int32_t b = 0; b < r.n_rb; ++b) {
    const RbRec nxt = recs[b + 1];
    const int32_t k0 = cur.k0, k1 = nxt.k0;
    if (k0 >= kcut) break;
    const float2 rho1 = rho_at(nxt, dC, dcst);
    const float2 slope = make_float2((rho1.x - rho.x) * cur.invw, (rho1.y - rho.y) * cur.invw);
    if (k1 <= kcut) {
      cmac(rho, make_float2(cur.sum.x, cur.sum.y), zr, zi);
      cmac(slope, make_float2(cur.sum.z, cur.sum.w), zr, zi);
      if ((b + 1) % kRbChunk == 0) {
        zr_all.add(zr);
        zi_all.add(zi);
        zr = zi = 0.f;
      }
    } else {
      // the bin holding the ISCO cut: its sums below the cut, from the prefix tables
      const int64_t m = (int64_t)a.n_bins + 1;
      const double* T = r.prefix;
      const double a0r = T[kcut] - T[k0], a0i = T[m + kcut] - T[m + k0];
      const double ofs = (double)k0 * a.df;
      const double a1r = (T[2 * m + kcut] - T[2 * m + k0]) - ofs * a0r;
      const double a1i = (T[3 * m + kcut] - T[3 * m + k0]) - ofs * a0i;
      zr64 += (double)rho.x * a0r - (double)rho.y * a0i + (double)slope.x * a1r - (double)slope.y * a1i;
      zi64 += (double)rho.x * a0i + (double)rho.y * a0r + (double)slope.x * a1i + (double)slope.y * a1r;
      break;
    }
    rho = rho1;
    cur = nxt;
  }
  zr_all.add(zr);
  zi_all.add(zi);
  zr64 += zr_all.value() * r.scale;
  zi64 += zi_all.value() * r.scale;
  const double z = ms.amp * hypot(zr64, zi64);
  const double H = ms.amp * ms.amp * a.tfold[kcut];
  double ll;
  if (a.marg == MBIS_MARG_PHASE)
    ll = log_i0(z) - 0.5 * H;
  else if (a.marg == (MBIS_MARG_PHASE | MBIS_MARG_DISTANCE))
    ll = log_distance_marginal_mixed(z, H, a.dist, a.glf);  // as the fused kernel
  else
    ll = ms.amp * zr64 - 0.5 * H;  // no marginalisation: Re (d|h) - <h|h> / 2
  a.out[s] = ll;
}

template <typename T>
void rfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

mbis_status rb_fail(mbis_ctx* c, mbis_status st, const std::string& msg) {
  c->err = msg;
  set_last_error(msg);
  return st;
}

}  // namespace

void rb_free(mbis_ctx* c) {
  rfree(c->d_rb_edges);
  rfree(c->d_rb_rec);
  rfree(c->d_rb_prefix);
  c->rb_n = 0;
}

}  // namespace mbis

using namespace mbis;

#define RB_TRY(c, call)                                                                           \
  do {                                                                                            \
    const cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                        \
      return rb_fail((c), e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,             \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

extern "C" {

mbis_status mbis_rb_setup(mbis_ctx* c, const double* theta0, int32_t n_rb, const int32_t* edges) {
  if (!c) {
    set_last_error("mbis_rb_setup: null context");
    return MBIS_E_INVALID;
  }
  if (!c->has_metric) return rb_fail(c, MBIS_E_STATE, "mbis_rb_setup: call mbis_set_metric first");
  if (c->tables_mode != 1)
    return rb_fail(c, MBIS_E_UNSUPPORTED, "mbis_rb_setup: relative binning needs fixed sky and orientation");
  if (c->opts.marg & MBIS_MARG_TIME)
    return rb_fail(c, MBIS_E_UNSUPPORTED, "mbis_rb_setup: time marginalisation is not supported");
  if (!theta0 || !edges || n_rb < 1 || n_rb > c->n_bins)
    return rb_fail(c, MBIS_E_INVALID, "mbis_rb_setup: need a fiducial and 1 <= n_rb <= n_bins edges");
  if (edges[0] != 0 || edges[n_rb] != c->n_bins)
    return rb_fail(c, MBIS_E_INVALID, "mbis_rb_setup: edges must run from 0 to n_bins");
  for (int32_t b = 0; b < n_rb; ++b)
    if (!(edges[b + 1] > edges[b])) return rb_fail(c, MBIS_E_INVALID, "mbis_rb_setup: edges must increase");
  if (!(theta0[kMc] > 0.0) || !(theta0[kQ] > 0.0))
    return rb_fail(c, MBIS_E_INVALID, "mbis_rb_setup: the fiducial needs Mc > 0 and q > 0");
  rb_free(c);
  const int32_t n = c->n_bins;
  const PhaseCoeffs pc0 = phase_coeffs(theta0[kMc], theta0[kQ], theta0[kChi1], theta0[kChi2], theta0[kTc],
                                       theta0[kPhic]);
  double* d_w = nullptr;
  double* d_max = nullptr;
  auto cleanup = [&]() {
    if (d_w) cudaFree(d_w);
    if (d_max) cudaFree(d_max);
  };
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMalloc(&d_w, sizeof(double) * 4 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_rb_prefix, sizeof(double) * 4 * ((size_t)n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_rb_edges, sizeof(int32_t) * (n_rb + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_rb_rec, sizeof(RbRec) * (n_rb + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_rb_edges, edges, sizeof(int32_t) * (n_rb + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    rb_weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, c->d_cfold64, c->d_basis, pc0, c->f_lo, c->df, d_w);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_prefix_rows(d_w, 4, n, c->d_rb_prefix, s);
  // the FP32 copies of the sums are scaled by a power of two near the largest bin sum
  std::vector<double> tot(4);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double mx = 0.0;
  if (e == cudaSuccess) {
    std::vector<double> T((size_t)4 * (n + 1));
    e = cudaMemcpy(T.data(), c->d_rb_prefix, sizeof(double) * T.size(), cudaMemcpyDeviceToHost);
    const int64_t m = (int64_t)n + 1;
    for (int32_t b = 0; b < n_rb && e == cudaSuccess; ++b) {
      const int32_t k0 = edges[b], k1 = edges[b + 1];
      mx = std::max(mx, std::hypot(T[k1] - T[k0], T[m + k1] - T[m + k0]));
    }
  }
  c->rb_scale = (mx > 0.0 && std::isfinite(mx)) ? std::ldexp(1.0, std::ilogb(mx) + 1) : 1.0;
  if (e == cudaSuccess) {
    rb_summary_kernel<<<(n_rb + 1 + 127) / 128, 128, 0, s>>>(n_rb, n, c->d_rb_edges, c->d_rb_prefix, c->f_lo,
                                                             c->df, 1.0 / c->rb_scale,
                                                             static_cast<RbRec*>(c->d_rb_rec));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) {
    rb_free(c);
    return rb_fail(c, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
                   std::string("mbis_rb_setup: ") + cudaGetErrorString(e));
  }
  for (int j = 0; j < kNumBasis; ++j) c->rb_C0[j] = pc0.C[j];
  c->rb_cst0 = pc0.cst;
  c->rb_n = n_rb;
  c->rb_gen = c->gen;
  return MBIS_OK;
}

mbis_status mbis_rb_loglike(mbis_ctx* c, int64_t n, const double* theta, double* loglike, void* stream) {
  if (!c) {
    set_last_error("mbis_rb_loglike: null context");
    return MBIS_E_INVALID;
  }
  if (c->rb_n == 0 || c->rb_gen != c->gen)
    return rb_fail(c, MBIS_E_STATE, "mbis_rb_loglike: call mbis_rb_setup (after the last mbis_set_metric)");
  if (n < 0 || (n > 0 && (!theta || !loglike))) return rb_fail(c, MBIS_E_INVALID, "mbis_rb_loglike: bad n or buffer");
  if (n == 0) return MBIS_OK;
  RbArgs r;
  r.la = make_like_args(c, n, theta, loglike);
  r.n_rb = c->rb_n;
  r.rec = static_cast<const RbRec*>(c->d_rb_rec);
  r.prefix = c->d_rb_prefix;
  r.scale = c->rb_scale;
  for (int j = 0; j < kNumBasis; ++j) r.C0[j] = c->rb_C0[j];
  r.cst0 = c->rb_cst0;
  // the records in shared memory when they fit (a few CTAs per SM still), else through L1
  const size_t sh = sizeof(RbRec) * (size_t)(c->rb_n + 1);
  r.rec_smem = sh <= kRbSmemMax ? 1 : 0;
  if (r.rec_smem && sh > 48 * 1024) {
    static bool attr = false;
    if (!attr) {
      RB_TRY(c, cudaFuncSetAttribute(rb_loglike_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRbSmemMax));
      attr = true;
    }
  }
  rb_loglike_kernel<<<(unsigned)((n + kRbThreads - 1) / kRbThreads), kRbThreads, r.rec_smem ? sh : 0,
                      static_cast<cudaStream_t>(stream)>>>(r);
  RB_TRY(c, cudaGetLastError());
  return MBIS_OK;
}

mbis_status mbis_rb_edges(const mbis_ctx* cc, const double* theta0, double n_sigma, double eps_rad, int32_t max_bins,
                          int32_t* edges, int32_t* n_rb) {
  mbis_ctx* c = const_cast<mbis_ctx*>(cc);
  if (!c) {
    set_last_error("mbis_rb_edges: null context");
    return MBIS_E_INVALID;
  }
  if (!c->has_metric) return rb_fail(c, MBIS_E_STATE, "mbis_rb_edges: call mbis_set_metric first");
  if (!theta0 || !edges || !n_rb || !(n_sigma > 0.0) || !(eps_rad > 0.0) || max_bins < 1)
    return rb_fail(c, MBIS_E_INVALID, "mbis_rb_edges: need a fiducial, n_sigma > 0, eps > 0, max_bins >= 1");
  // largest coefficient offsets over the corners of the box theta0 +- n_sigma proposal
  // sigmas (clipped to the prior), every sampled slot at once
  const int P = c->P;
  double sig[kMaxP];
  for (int p = 0; p < P; ++p) {
    double v = 0.0;
    for (int r = 0; r <= p; ++r) v += c->chol[p * kMaxP + r] * c->chol[p * kMaxP + r];
    sig[p] = n_sigma * c->scale * std::sqrt(v);
  }
  const PhaseCoeffs pc0 = phase_coeffs(theta0[kMc], theta0[kQ], theta0[kChi1], theta0[kChi2], theta0[kTc],
                                       theta0[kPhic]);
  double dC[kNumBasis] = {};
  for (int mask = 0; mask < (1 << P); ++mask) {
    double th[kNumSlots];
    std::memcpy(th, theta0, sizeof(th));
    for (int p = 0; p < P; ++p) {
      const int id = c->ids[p];
      double v = theta0[id] + ((mask >> p) & 1 ? sig[p] : -sig[p]);
      v = std::min(std::max(v, c->lo[p]), c->hi[p]);
      th[id] = v;
    }
    if (!(th[kMc] > 0.0) || !(th[kQ] > 0.0)) continue;
    const PhaseCoeffs pc = phase_coeffs(th[kMc], th[kQ], th[kChi1], th[kChi2], th[kTc], th[kPhic]);
    for (int j = 0; j < kNumBasis; ++j) dC[j] = std::max(dC[j], std::fabs(pc.C[j] - pc0.C[j]));
  }
  // greedy bins: the largest change of the phase difference across a bin stays below eps
  // (a single grid step is the narrowest bin); the last edge is n_bins
  const int32_t n = c->n_bins;
  int32_t nb = 0, k0 = 0;
  edges[0] = 0;
  double b0[kNumBasis];
  auto load_b0 = [&]() {
    for (int j = 0; j < kNumBasis; ++j) b0[j] = basis(j, c->f_lo + (double)k0 * c->df);
  };
  load_b0();
  for (int32_t k = 1; k < n; ++k) {
    const double f = c->f_lo + (double)k * c->df;
    double dphi = 0.0;
    for (int j = 0; j < kNumBasis; ++j) dphi += dC[j] * std::fabs(basis(j, f) - b0[j]);
    if (kTwoPi * dphi > eps_rad && k - 1 > k0) {
      if (nb + 1 >= max_bins) return rb_fail(c, MBIS_E_INVALID, "mbis_rb_edges: more bins than max_bins");
      edges[++nb] = k - 1;
      k0 = k - 1;
      load_b0();
      --k;  // test this grid point again from the new edge
    }
  }
  edges[++nb] = n;
  *n_rb = nb;
  return MBIS_OK;
}

}  // extern "C"
