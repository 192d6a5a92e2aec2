// k_rb.cu -- relative binning (the heterodyned likelihood of Zackay, Dai & Venumadhav 2018;
// the paper notes that faster likelihoods such as this plug into its method, Sec. IV) for
// contexts whose extrinsic parameters are fixed, so that the detectors fold into one table.
//
// About a fiducial theta0 the template's ratio to the fiducial, r(f) = (A / A0)
// e^(-i 2 pi (Psi(f) - Psi0(f))), is smooth; inside each coarse bin [f_b, f_b+1) it is
// replaced by its chord through the bin's edges.  With the fiducial-heterodyned data weights
// W_k = c_k e^(-i 2 pi Psi0(f_k)) (c the folded data table, which carries the detector
// responses, delays, f^(-7/6), 1/S and 4 df), the overlap becomes
//   Z = A sum_b [rho_b A0_b + (rho_b+1 - rho_b) / (f_b+1 - f_b) A1_b],
//   A0_b = sum_{k in b} W_k,  A1_b = sum_{k in b} W_k (f_k - f_b),  rho_e = e^(-i 2 pi dPsi(f_e)).
// Regrouped by edge, with p_b = A0_b - A1_b / w_b and q_b = A1_b / w_b (w_b the bin's width),
//   Z = A [sum_{e < n} rho_e (p_e + q_e-1) + rho_n q_n-1],
// n the number of bins that lie wholly below the sample's ISCO cut: one complex weight per
// edge, so that the sweep costs one phase evaluation and one complex multiply-add per edge.
// The bin holding the cut is summed only below it (from FP64 prefix sums); <h|h> stays exact
// (the amplitude prefix table).  The phase difference from the fiducial's runs in FP32 from
// FP64 coefficient differences, then MUFU sine / cosine; the edge sums run in FP32 over
// chunks of 16 edges whose sums are gathered as float pairs (no FP64 arithmetic in the
// sweep).
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

constexpr int kRbThreads = 256;
constexpr int kRbChunk = 16;
constexpr size_t kRbSmemMax = 112 * 1024;  // records staged in shared memory up to 2388 bins
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

// One edge record: three float4 = (c_e re, c_e im, B_0, B_1), (B_2 .. B_5), (B_6, B_7, B_8, 0),
// c_e = (p_e + q_e-1) / scale (zero at the last edge) and B_j the basis at the edge.
constexpr int kEdgeVec = 3;

// bin b's sums from the prefix tables: A0 and A1 / w as (re, im) pairs
__device__ __forceinline__ void bin_sums(const double* T, int64_t m, int32_t k0, int32_t k1, double df, double& a0r,
                                         double& a0i, double& qr, double& qi) {
  a0r = T[k1] - T[k0];
  a0i = T[m + k1] - T[m + k0];
  const double ofs = (double)k0 * df;  // f_b - f_lo
  const double inv_w = 1.0 / ((double)(k1 - k0) * df);
  qr = ((T[2 * m + k1] - T[2 * m + k0]) - ofs * a0r) * inv_w;
  qi = ((T[3 * m + k1] - T[3 * m + k0]) - ofs * a0i) * inv_w;
}

__global__ void rb_summary_kernel(int32_t n_rb, int32_t n, const int32_t* __restrict__ edges,
                                  const double* __restrict__ T, double f_lo, double df, double inv_scale,
                                  float4* rec, float2* q_out) {
  const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > n_rb) return;
  const int64_t m = (int64_t)n + 1;
  double cr = 0.0, ci = 0.0;
  if (e < n_rb) {
    double a0r, a0i, qr, qi;
    bin_sums(T, m, edges[e], edges[e + 1], df, a0r, a0i, qr, qi);
    cr += a0r - qr;
    ci += a0i - qi;
    q_out[e] = make_float2((float)(qr * inv_scale), (float)(qi * inv_scale));
  }
  if (e > 0 && e < n_rb) {
    double a0r, a0i, qr, qi;
    bin_sums(T, m, edges[e - 1], edges[e], df, a0r, a0i, qr, qi);
    cr += qr;
    ci += qi;
  }
  float b[kNumBasis];
  const double fe = f_lo + (double)edges[e] * df;
  for (int j = 0; j < kNumBasis; ++j) b[j] = (float)basis(j, fe);
  float4* r = rec + (int64_t)kEdgeVec * e;
  r[0] = make_float4((float)(cr * inv_scale), (float)(ci * inv_scale), b[0], b[1]);
  r[1] = make_float4(b[2], b[3], b[4], b[5]);
  r[2] = make_float4(b[6], b[7], b[8], 0.0f);
}

struct RbArgs {
  LikeArgs la;
  int32_t n_rb;
  const float4* rec;     // [n_rb + 1][kEdgeVec]
  const float2* q;       // [n_rb] q_b / scale
  const int32_t* edges;  // [n_rb + 1]
  int32_t rec_smem;      // stage the records in shared memory
  const double* prefix;  // [4][n_bins + 1]
  double scale;
  double C0[kNumBasis], cst0;
};

// e^(-i 2 pi dPsi) at one edge, and the edge's weight c_e
__device__ __forceinline__ float2 edge_rho(const float4* __restrict__ e, const float* dC, float dcst, float2& c) {
  const float4 r0 = e[0], r1 = e[1], r2 = e[2];
  c = make_float2(r0.x, r0.y);
  float t = fmaf(dC[0], r0.z, dcst);
  t = fmaf(dC[1], r0.w, t);
  t = fmaf(dC[2], r1.x, t);
  t = fmaf(dC[3], r1.y, t);
  t = fmaf(dC[4], r1.z, t);
  t = fmaf(dC[5], r1.w, t);
  t = fmaf(dC[6], r2.x, t);
  t = fmaf(dC[7], r2.y, t);
  t = fmaf(dC[8], r2.z, t);
  // the nearest integer removed (1.5 * 2^23 rounds |t| < 2^22 to an integer): turns in [-1/2, 1/2]
  t = __fsub_rn(t, __fsub_rn(__fadd_rn(t, 12582912.0f), 12582912.0f));
  float s, co;
  __sincosf(-kTwoPiF * t, &s, &co);
  return make_float2(co, s);
}

__global__ void __launch_bounds__(kRbThreads, 3) rb_loglike_kernel(RbArgs r) {
  extern __shared__ float4 s_rec[];
  const LikeArgs& a = r.la;
  const float4* recs = r.rec;
  if (r.rec_smem) {
    for (int i = threadIdx.x; i < kEdgeVec * (r.n_rb + 1); i += blockDim.x) s_rec[i] = __ldg(r.rec + i);
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
  const SampleSetup ss = sample_setup(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic], dl, a.f_lo,
                                      a.df, a.n_bins);
  const PhaseCoeffs& pc = ss.pc;
  const int32_t kcut = ss.kcut;
  const double amp = ss.amp;
  float dC[kNumBasis];
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) dC[j] = (float)(pc.C[j] - r.C0[j]);
  const float dcst = (float)(pc.cst - r.cst0);

  // nfull = the last edge at or below the cut: bins 0 .. nfull-1 lie wholly below it
  int32_t lo = 0, hi = r.n_rb;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(r.edges + mid) <= kcut)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int32_t nfull = lo;

  FFSum zr_all, zi_all;  // chunk sums, scaled by 1 / scale
  int32_t e = 0;
  for (; e + kRbChunk <= nfull; e += kRbChunk) {
    float zr = 0.f, zi = 0.f;
#pragma unroll
    for (int j = 0; j < kRbChunk; ++j) {
      float2 c;
      const float2 rho = edge_rho(recs + kEdgeVec * (e + j), dC, dcst, c);
      zr = fmaf(rho.x, c.x, fmaf(-rho.y, c.y, zr));
      zi = fmaf(rho.x, c.y, fmaf(rho.y, c.x, zi));
    }
    zr_all.add(zr);
    zi_all.add(zi);
  }
  float zr = 0.f, zi = 0.f;
  for (; e < nfull; ++e) {
    float2 c;
    const float2 rho = edge_rho(recs + kEdgeVec * e, dC, dcst, c);
    zr = fmaf(rho.x, c.x, fmaf(-rho.y, c.y, zr));
    zi = fmaf(rho.x, c.y, fmaf(rho.y, c.x, zi));
  }
  // edge nfull: the far end of the last whole bin, and the near end of the bin holding the cut
  float2 c_unused;
  const float2 rho_n = edge_rho(recs + kEdgeVec * nfull, dC, dcst, c_unused);
  if (nfull > 0) {
    const float2 q = r.q[nfull - 1];
    zr = fmaf(rho_n.x, q.x, fmaf(-rho_n.y, q.y, zr));
    zi = fmaf(rho_n.x, q.y, fmaf(rho_n.y, q.x, zi));
  }
  zr_all.add(zr);
  zi_all.add(zi);
  double zr64 = zr_all.value() * r.scale, zi64 = zi_all.value() * r.scale;
  const int32_t k0 = __ldg(r.edges + nfull);
  if (k0 < kcut) {
    // the bin holding the ISCO cut (nfull < n_rb here): its sums below the cut, from the
    // prefix tables, against the chord through the bin's two edges
    const int32_t k1 = __ldg(r.edges + nfull + 1);
    const float2 rho1 = edge_rho(recs + kEdgeVec * (nfull + 1), dC, dcst, c_unused);
    const double inv_w = 1.0 / ((double)(k1 - k0) * a.df);
    const double sr = (double)(rho1.x - rho_n.x) * inv_w, si = (double)(rho1.y - rho_n.y) * inv_w;
    const int64_t m = (int64_t)a.n_bins + 1;
    const double* T = r.prefix;
    const double a0r = T[kcut] - T[k0], a0i = T[m + kcut] - T[m + k0];
    const double ofs = (double)k0 * a.df;
    const double a1r = (T[2 * m + kcut] - T[2 * m + k0]) - ofs * a0r;
    const double a1i = (T[3 * m + kcut] - T[3 * m + k0]) - ofs * a0i;
    zr64 += (double)rho_n.x * a0r - (double)rho_n.y * a0i + sr * a1r - si * a1i;
    zi64 += (double)rho_n.x * a0i + (double)rho_n.y * a0r + sr * a1i + si * a1r;
  }
  const double z = amp * hypot(zr64, zi64);
  const double H = amp * amp * a.tfold[kcut];
  double ll;
  if (a.marg == MBIS_MARG_PHASE)
    ll = log_i0(z) - 0.5 * H;
  else if (a.marg == (MBIS_MARG_PHASE | MBIS_MARG_DISTANCE))
    ll = log_distance_marginal_mixed(z, H, a.dist, a.glf);  // as the fused kernel
  else
    ll = amp * zr64 - 0.5 * H;  // no marginalisation: Re (d|h) - <h|h> / 2
  a.out[s] = ll;
}

mbis_status rb_fail(mbis_ctx* c, mbis_status st, const std::string& msg) {
  c->err = msg;
  set_last_error(msg);
  return st;
}

}  // namespace

void rb_free(mbis_ctx* c) {
  c->rb_use = 0;
  dfree(c, c->d_rb_edges);
  dfree(c, c->d_rb_rec);
  dfree(c, c->d_rb_q);
  dfree(c, c->d_rb_prefix);
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
  // device memory from the context's allocator (stream-ordered from its pool when it has
  // one, as in the request server), copies on its stream
  double* d_w = nullptr;
  cudaStream_t s = c->stream;
  cudaError_t e = dalloc(c, &d_w, sizeof(double) * 4 * (size_t)n);
  if (e == cudaSuccess) e = dalloc(c, &c->d_rb_prefix, sizeof(double) * 4 * ((size_t)n + 1));
  if (e == cudaSuccess) e = dalloc(c, &c->d_rb_edges, sizeof(int32_t) * (n_rb + 1));
  if (e == cudaSuccess) e = dalloc(c, &c->d_rb_rec, sizeof(float4) * kEdgeVec * (n_rb + 1));
  if (e == cudaSuccess) e = dalloc(c, &c->d_rb_q, sizeof(float2) * n_rb);
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
    e = cudaMemcpyAsync(T.data(), c->d_rb_prefix, sizeof(double) * T.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
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
                                                             static_cast<float4*>(c->d_rb_rec),
                                                             static_cast<float2*>(c->d_rb_q));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(c, d_w);
  if (e != cudaSuccess) {
    rb_free(c);
    return rb_fail(c, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
                   std::string("mbis_rb_setup: ") + cudaGetErrorString(e));
  }
  for (int j = 0; j < kNumBasis; ++j) c->rb_C0[j] = pc0.C[j];
  c->rb_cst0 = pc0.cst;
  c->rb_n = n_rb;
  c->rb_gen = c->tables_gen;
  return MBIS_OK;
}

mbis_status mbis_rb_loglike(mbis_ctx* c, int64_t n, const double* theta, double* loglike, void* stream) {
  if (!c) {
    set_last_error("mbis_rb_loglike: null context");
    return MBIS_E_INVALID;
  }
  if (c->rb_n == 0 || c->rb_gen != c->tables_gen)
    return rb_fail(c, MBIS_E_STATE, "mbis_rb_loglike: call mbis_rb_setup (after the last mbis_set_metric)");
  if (n < 0 || (n > 0 && (!theta || !loglike))) return rb_fail(c, MBIS_E_INVALID, "mbis_rb_loglike: bad n or buffer");
  if (n == 0) return MBIS_OK;
  RbArgs r;
  r.la = make_like_args(c, n, theta, loglike);
  r.n_rb = c->rb_n;
  r.rec = static_cast<const float4*>(c->d_rb_rec);
  r.q = static_cast<const float2*>(c->d_rb_q);
  r.edges = c->d_rb_edges;
  r.prefix = c->d_rb_prefix;
  r.scale = c->rb_scale;
  for (int j = 0; j < kNumBasis; ++j) r.C0[j] = c->rb_C0[j];
  r.cst0 = c->rb_cst0;
  // the records in shared memory when they fit (a few CTAs per SM still), else through L1
  const size_t sh = sizeof(float4) * kEdgeVec * (size_t)(c->rb_n + 1);
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

mbis_status mbis_rb_use(mbis_ctx* c, int32_t on) {
  if (!c) {
    set_last_error("mbis_rb_use: null context");
    return MBIS_E_INVALID;
  }
  if (on && (c->rb_n == 0 || c->rb_gen != c->tables_gen))
    return rb_fail(c, MBIS_E_STATE, "mbis_rb_use: call mbis_rb_setup (after the last mbis_set_metric)");
  c->rb_use = on ? 1 : 0;
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
  double b0[kNumBasis], bk[kNumBasis];
  auto load_b0 = [&]() { basis_all(c->f_lo + (double)k0 * c->df, b0); };
  load_b0();
  for (int32_t k = 1; k < n; ++k) {
    basis_all(c->f_lo + (double)k * c->df, bk);
    double dphi = 0.0;
    for (int j = 0; j < kNumBasis; ++j) dphi += dC[j] * std::fabs(bk[j] - b0[j]);
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
