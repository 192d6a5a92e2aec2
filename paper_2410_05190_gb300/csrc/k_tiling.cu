// k_tiling.cu -- kernels of the tiled proposal (Sec. II; App. A): FP64 waveforms and
// matches for template placement, the tensor-core tile assignment of prior samples, the
// stable per-tile member lists, the mixture over tiles and its draws.
//
// Waveforms are the TaylorF2 model of the likelihood (physics.cuh) at zero coalescence
// time and phase, whitened by one PSD and scaled to unit norm:
//   u_k = w_k e^(-i Psi(f_k)) / sqrt(sum_{k' < kcut} w_k'^2),  w_k = f_k^(-7/6) / sqrt(S_k),
// zero at and above the ISCO.  The match of two points is |sum_k conj(u_a,k) u_b,k|, the
// normalised overlap maximised over a constant phase.
#include <cuda_fp16.h>

#include "physics.cuh"
#include "philox.cuh"
#include "tc.cuh"
#include "tiling.h"

namespace mbis {
namespace {

__host__ __device__ inline void map_point(const TilingSpace& sp, double x, double q, double& mc, double& qp) {
  if (sp.mc_period > 0.0) {
    double r = fmod(x, sp.mc_period);
    if (r < 0.0) r += sp.mc_period;
    mc = sp.mc_base + r;
  } else {
    mc = x;
  }
  qp = q >= 1.0 ? q : 1.0 / q;
}

__device__ __forceinline__ bool in_space(const TilingSpace& sp, double x, double q) {
  return x >= sp.x_lo && x < sp.x_hi && q >= sp.q_lo && q <= sp.q_hi;
}

// FP64 phase (turns) of a point's coefficients at frequency f
__device__ __forceinline__ double phase_turns(const PhaseCoeffs& pc, double f) {
  double t = pc.cst;
#pragma unroll
  for (int j = 0; j < kNumBasis - 1; ++j) t = fma(pc.C[j], basis(j, f), t);
  return t;  // C[8] multiplies f: the coalescence time, zero here
}

struct PointSetup {
  PhaseCoeffs pc;
  int32_t kcut;
  double inv_norm;
};

__device__ __forceinline__ PointSetup point_setup(const TilingSpace& sp, const TilingGrid& g, double x, double q) {
  PointSetup o;
  double mc, qp;
  map_point(sp, x, q, mc, qp);
  const double m_sec = total_mass_seconds(mc, qp);
  o.pc = phase_coeffs_m(mc, qp, sp.chi1, sp.chi2, 0.0, 0.0, m_sec);
  o.kcut = live_bins_m(m_sec, g.f_lo, g.df, g.K);
  o.inv_norm = o.kcut > 0 ? 1.0 / sqrt(g.w2sum[o.kcut]) : 0.0;
  return o;
}

// ---- FP64 waveforms, one CTA per point -------------------------------------------------
__global__ void waveforms_kernel(TilingSpace sp, TilingGrid g, int32_t n, const double* __restrict__ pts,
                                 double2* rows, double2* kmaj, int32_t ldk, int32_t col0) {
  const int32_t p = blockIdx.x;
  if (p >= n) return;
  const PointSetup ps = point_setup(sp, g, pts[p], pts[n + p]);
  for (int32_t k = threadIdx.x; k < g.K; k += blockDim.x) {
    double2 u = make_double2(0.0, 0.0);
    if (k < ps.kcut) {
      double t = phase_turns(ps.pc, g.f_lo + (double)k * g.df);
      t -= floor(t);
      double s, c;
      sincospi(2.0 * t, &s, &c);
      const double a = g.w[k] * ps.inv_norm;
      u = make_double2(a * c, -a * s);
    }
    if (rows) rows[(int64_t)p * g.K + k] = u;
    if (kmaj) kmaj[(int64_t)k * ldk + col0 + p] = u;
  }
}

// ---- FP64 |conj(A) . B| for template placement ----------------------------------------
// A CTA holds kDotRows rows of A in shared memory, kDotChunk bins at a time, and each
// thread one column of B (k-major, so a warp's loads of one bin are contiguous); the sum
// over bins runs in bin order.
constexpr int kDotRows = 32, kDotChunk = 32, kDotThreads = 128;

__global__ void __launch_bounds__(kDotThreads) absdots_kernel(int32_t na, const double2* __restrict__ A, int32_t nb,
                                                              const double2* __restrict__ B, int32_t ldb, int32_t K,
                                                              double* __restrict__ out) {
  __shared__ double2 sa[kDotRows][kDotChunk];
  const int32_t j = blockIdx.x * kDotThreads + threadIdx.x;
  const int32_t i0 = blockIdx.y * kDotRows;
  double zr[kDotRows], zi[kDotRows];
#pragma unroll
  for (int r = 0; r < kDotRows; ++r) zr[r] = zi[r] = 0.0;
  for (int32_t k0 = 0; k0 < K; k0 += kDotChunk) {
    __syncthreads();
    for (int e = threadIdx.x; e < kDotRows * kDotChunk; e += kDotThreads) {
      const int r = e / kDotChunk, kk = e % kDotChunk;
      const int32_t i = i0 + r, k = k0 + kk;
      sa[r][kk] = (i < na && k < K) ? A[(int64_t)i * K + k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (j < nb) {
      const int kn = min(kDotChunk, K - k0);
      for (int kk = 0; kk < kn; ++kk) {
        const double2 b = B[(int64_t)(k0 + kk) * ldb + j];
#pragma unroll
        for (int r = 0; r < kDotRows; ++r) {
          const double2 a = sa[r][kk];
          zr[r] = fma(a.y, b.y, fma(a.x, b.x, zr[r]));   // Re conj(a) b
          zi[r] = fma(-a.y, b.x, fma(a.x, b.y, zi[r]));  // Im conj(a) b
        }
      }
    }
  }
  if (j < nb) {
#pragma unroll
    for (int r = 0; r < kDotRows; ++r)
      if (i0 + r < na) out[(int64_t)(i0 + r) * nb + j] = sqrt(zr[r] * zr[r] + zi[r] * zi[r]);
  }
}

// ---- FP64 match of point pairs, one warp per pair --------------------------------------
__global__ void pair_match_kernel(TilingSpace sp, TilingGrid g, int64_t n, const double* __restrict__ a,
                                  const double* __restrict__ b, double* __restrict__ out) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n) return;
  const PointSetup sa = point_setup(sp, g, a[p], a[n + p]);
  const PointSetup sb = point_setup(sp, g, b[p], b[n + p]);
  const int32_t kc = min(sa.kcut, sb.kcut);
  double zr = 0.0, zi = 0.0;
  for (int32_t k = lane; k < kc; k += 32) {
    const double f = g.f_lo + (double)k * g.df;
    double d = phase_turns(sa.pc, f) - phase_turns(sb.pc, f);  // conj(u_a) u_b ~ e^(+i (Psi_a - Psi_b))
    d -= floor(d);
    double s, c;
    sincospi(2.0 * d, &s, &c);
    const double w2 = g.w[k] * g.w[k];
    zr = fma(w2, c, zr);
    zi = fma(w2, s, zi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    zr += __shfl_xor_sync(0xffffffffu, zr, o);
    zi += __shfl_xor_sync(0xffffffffu, zi, o);
  }
  if (lane == 0) out[p] = (kc > 0) ? sqrt(zr * zr + zi * zi) * sa.inv_norm * sb.inv_norm : 0.0;
}

__global__ void append_kernel(int32_t n, const int32_t* __restrict__ idx, const double2* __restrict__ src, int32_t K,
                              double2* dst_rows, int32_t row0, double2* dst_kmaj, int32_t ldk) {
  const int32_t i = blockIdx.x;
  if (i >= n) return;
  const double2* s = src + (int64_t)idx[i] * K;
  for (int32_t k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = s[k];
    dst_rows[(int64_t)(row0 + i) * K + k] = v;
    dst_kmaj[(int64_t)k * ldk + row0 + i] = v;
  }
}

// ---- FP32 tables of the tensor-core pass -----------------------------------------------
// Record of bin pair p (bins 2p, 2p + 1): basis_j at both bins for j = 0..7 as pairs,
// then the two whitening weights scaled by wscale = 1 / max(w), then padding.
__global__ void bin_records_kernel(TilingGrid g, double wscale, float* out) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n_kb * (kTileBins / 2)) return;
  float* r = out + (int64_t)p * kBinRecord;
  for (int e = 0; e < 2; ++e) {
    const int32_t k = 2 * p + e;
    const double f = g.f_lo + (double)k * g.df;
    for (int j = 0; j < kNumBasis - 1; ++j) r[2 * j + e] = (float)basis(j, f);
    r[16 + e] = k < g.K ? (float)(g.w[k] * wscale) : 0.f;
  }
  r[18] = 0.f;
  r[19] = 0.f;
}

// Template operand: pass p holds templates perm[256 p .. 256 p + 255] (ordered by live-bin
// count; -1 pads), as two halves of 128 templates, each 256 rows (template slot i: row 2i
// gives Re conj(a) b, row 2i + 1 Im conj(a) b against a sample row laid out as
// (Re a_k, Im a_k) pairs), one 32-bin K-block of 64 FP16 values per 128-byte row, 16-byte
// chunk c of row n at byte n * 128 + ((c ^ (n & 7)) << 4) (the 128-byte swizzle).
// Layout [pass][K-block][half][256 rows][64].
__global__ void template_tiles_kernel(const int32_t* __restrict__ perm, const double2* __restrict__ rows, TilingGrid g,
                                      __half* out) {
  const int32_t kb = blockIdx.x, ph = blockIdx.y, n = threadIdx.x;
  const int32_t p = ph >> 1, h = ph & 1;
  const int32_t t = perm[p * 2 * kTileTemplates + h * kTileTemplates + (n >> 1)];
  const bool im = n & 1;
  __half* tile = out + (((int64_t)p * g.n_kb + kb) * 2 + h) * (kTileBytes / 2);
  for (int kk = 0; kk < kTileBins; ++kk) {
    const int32_t k = kb * kTileBins + kk;
    double2 v = make_double2(0.0, 0.0);
    if (t >= 0 && k < g.K) v = rows[(int64_t)t * g.K + k];
    const float e[2] = {(float)(im ? v.y : v.x), (float)(im ? -v.x : v.y)};
    for (int c = 0; c < 2; ++c) {
      const int kidx = 2 * kk + c, c16 = kidx >> 3, pos = kidx & 7;
      tile[n * 64 + (((c16 ^ (n & 7)) << 3) | pos)] = __float2half_rn(e[c]);
    }
  }
}

// ---- tile assignment on the tensor cores ------------------------------------------------
// The sample-by-template overlaps are a real contraction [samples x 2K] . [2K x 2T].  A CTA
// owns 128 samples (the MMA's M) and visits the templates in passes of 256: two MMA column
// blocks of N = 256 (128 templates each as Re / Im rows), accumulated in TMEM columns
// [0, 256) and [256, 512).  Templates are ordered by live-bin count and each pass runs only
// over the K-blocks that both its templates and the CTA's samples reach.  Operands are FP16
// (the 11-bit significand of TF32 at twice its rate and half its bytes; the normalised
// waveform values, ~0.1, sit far inside the FP16 range).  Sixteen compute warps write the
// sample operand: per 32-bin K-block, four threads per sample (one per 8-bin quarter)
// compute e^(-i Psi) of their bins from FP32 phase coefficients and write them, rounded to
// FP16, into the sample's row of a 128-byte-swizzled shared-memory tile.  A seventeenth warp
// issues the 2 x 4 tcgen05.mma.kind::f16 of each block once its operands are in place,
// commits to an mbarrier, and bulk-copies the next block's template tile.  After a pass's
// last block each compute thread reads back 64 of its sample's 256 complex overlaps (one
// block late, before the next pass's first MMA overwrites them) and keeps the running best;
// the four parts' bests are merged at the end.
constexpr int kParts = 4;                        // threads per sample
constexpr int kACompute = 128 * kParts;          // compute threads
constexpr int kAThreads = kACompute + 32;        // + the MMA-issuer warp
constexpr uint32_t kATile = 16384;               // 128 rows x 128 bytes
constexpr uint32_t kBHalf = kTileBytes;          // 256 rows (128 templates) x 128 bytes
constexpr uint32_t kBBlock = 2 * kBHalf;         // one K-block of a pass
constexpr uint32_t kAOffA = 0;                   // [2 buf][kATile]
constexpr uint32_t kAOffB = kAOffA + 2 * kATile; // [2 buf][kBBlock]
constexpr uint32_t kAOffR = kAOffB + 2 * kBBlock;  // basis records of the CTA's bins
constexpr uint32_t kRecSmem = 24576;             // up to 19 K-blocks (608 bins) of records
constexpr uint32_t kASmem = kAOffR + kRecSmem + 1024;
constexpr uint32_t kAIdesc = tc::idesc_f16(128, 2 * kTileTemplates);
constexpr float kTwoPiF = 6.28318530717958647692f;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The TaylorF2 phase coefficients of physics.cuh (phase_coeffs_a, the same series) in
// single precision, for the FP16 sample operand: q >= 1, a = pi M, la = ln a, a13 = a^(1/3);
// C[j] in turns for basis j = 0..7 (the constant and the coalescence-time term drop out of
// the match).  The constants are folded in double at compile time.
__device__ __forceinline__ void phase_coeffs_f32(float q, float chi1, float chi2, float a, float la, float a13,
                                                 float* C) {
  constexpr float pi = (float)kPi;
  const float eta = q / ((1.f + q) * (1.f + q));
  const float dm = (q - 1.f) / (q + 1.f);
  const float xs = 0.5f * (chi1 + chi2), xa = 0.5f * (chi1 - chi2);
  const float e2 = eta * eta, e3 = e2 * eta;
  const float phi2 = (float)(3715.0 / 756.0) + (float)(55.0 / 9.0) * eta;
  const float phi3 = -16.f * pi + (float)(113.0 / 3.0) * dm * xa + ((float)(113.0 / 3.0) - (float)(76.0 / 3.0) * eta) * xs;
  const float phi4 = (float)(15293365.0 / 508032.0) + (float)(27145.0 / 504.0) * eta + (float)(3085.0 / 72.0) * e2 +
                     (-50.625f + 200.f * eta) * xa * xa - 101.25f * dm * xa * xs + (-50.625f + 2.5f * eta) * xs * xs;
  const float c5 = pi * ((float)(38645.0 / 756.0) - (float)(65.0 / 9.0) * eta) +
                   dm * ((float)(-732985.0 / 2268.0) - (float)(140.0 / 9.0) * eta) * xa +
                   ((float)(-732985.0 / 2268.0) + (float)(24260.0 / 81.0) * eta + (float)(340.0 / 9.0) * e2) * xs;
  const float a6 = (float)(11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi -
                           6848.0 / 21.0 * (kEulerGamma + 1.3862943611198906)) +
                   (float)(-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) * eta +
                   (float)(76055.0 / 1728.0) * e2 - (float)(127825.0 / 1296.0) * e3 +
                   pi * ((float)(2270.0 / 3.0) * dm * xa + ((float)(2270.0 / 3.0) - 520.f * eta) * xs) +
                   ((float)(75515.0 / 144.0) - (float)(8225.0 / 18.0) * eta) * dm * xa * xs +
                   ((float)(75515.0 / 288.0) - (float)(263245.0 / 252.0) * eta - 480.f * e2) * xa * xa +
                   ((float)(75515.0 / 288.0) - (float)(232415.0 / 504.0) * eta + (float)(1255.0 / 9.0) * e2) * xs * xs;
  const float phi7 =
      pi * ((float)(77096675.0 / 254016.0) + (float)(378515.0 / 1512.0) * eta - (float)(74045.0 / 756.0) * e2) +
      ((float)(-25150083775.0 / 3048192.0) + (float)(10566655595.0 / 762048.0) * eta -
       (float)(1042165.0 / 3024.0) * e2 + (float)(5345.0 / 36.0) * e3) * xs +
      dm * ((float)(-25150083775.0 / 3048192.0) + (float)(26804935.0 / 6048.0) * eta - (float)(1985.0 / 48.0) * e2) *
          xa;
  const float a23 = a13 * a13;
  const float pre = (float)(3.0 / 128.0 / kTwoPi) / eta;
  C[0] = pre / (a23 * a23 * a13);
  C[1] = pre * phi2 / a;
  C[2] = pre * phi3 / a23;
  C[3] = pre * phi4 / a13;
  C[4] = pre * c5;
  C[5] = pre * a13 * (a6 - (float)(6848.0 / 63.0) * la);
  C[6] = -pre * a13 * (float)(6848.0 / 63.0);
  C[7] = pre * phi7 * a23;
}

// Per-sample set-up of the FP16 operand: the live-bin count from the total mass in FP64
// (FP32 seed, one Newton step: the ISCO cut agrees with FP64 to the bin), the phase
// coefficients in FP32, the inverse norm from the FP64 prefix table.
struct FastSetup {
  float cf[kNumBasis - 1];
  int32_t kcut;
  float inv_s;
};

__device__ __forceinline__ FastSetup fast_setup(const TilingSpace& sp, const TilingGrid& g, double x, double q) {
  FastSetup o;
  double mc, qp;
  map_point(sp, x, q, mc, qp);
  const double u = (1.0 + qp) * (1.0 + qp) / qp, u3 = u * u * u;
  double y = (double)powf((float)u, 0.6f);
  const double y4 = (y * y) * (y * y);
  y = 0.8 * y + u3 / (5.0 * y4);                   // y^5 = u^3
  const double m_sec = mc * kTsun * y;
  o.kcut = live_bins_m(m_sec, g.f_lo, g.df, g.K);
  const float am = (float)(kPi * m_sec);
  phase_coeffs_f32((float)qp, (float)sp.chi1, (float)sp.chi2, am, logf(am), cbrtf(am), o.cf);
  o.inv_s = o.kcut > 0 ? rsqrtf((float)(g.w2sum[o.kcut] * g.inv_wref2)) : 0.f;
  return o;
}

// Set-up of every point at full occupancy: its record (FP32 phase coefficients, inverse
// norm, live-bin count; zero outside the space) and its live-bin count, the key that
// orders samples so that a CTA's samples reach similar K.
__global__ void setup_kernel(TilingSpace sp, TilingGrid g, int64_t n, const double* __restrict__ pts,
                             float4* __restrict__ rec, int32_t* __restrict__ kc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pts[i], q = pts[n + i];
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
  int32_t k = 0;
  if (in_space(sp, x, q)) {
    const FastSetup fs = fast_setup(sp, g, x, q);
    k = fs.kcut;
    r0 = make_float4(fs.cf[0], fs.cf[1], fs.cf[2], fs.cf[3]);
    r1 = make_float4(fs.cf[4], fs.cf[5], fs.cf[6], fs.cf[7]);
    r2 = make_float4(fs.inv_s, __int_as_float(k), 0.f, 0.f);
  }
  rec[3 * i] = r0;
  rec[3 * i + 1] = r1;
  rec[3 * i + 2] = r2;
  kc[i] = k;
}

__global__ void __launch_bounds__(kAThreads, 1) assign_kernel(AssignArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // bbar[b]: template tile of buffer b landed; full[b]: the 256 compute threads wrote A[b];
  // mbar[b]: the MMAs reading buffers b completed.
  __shared__ __align__(8) uint64_t bbar[2], full[2], mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_kmax, s_nblk;
  __shared__ int s_issued_b[2], s_issued_m[2];
  __shared__ volatile int s_bad;
  __shared__ float s_cf[kNumBasis - 1][128];
  __shared__ float s_inv[128];
  __shared__ int32_t s_kcut[128];
  __shared__ float s_b2[kParts][128];
  __shared__ int32_t s_bt[kParts][128];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool compute = tid < kACompute;
  const int row = tid & 127, part = compute ? tid >> 7 : 0;
  const int64_t slot = (int64_t)blockIdx.x * 128 + row;
  const bool active = compute && slot < a.n;
  const int64_t s = active ? (a.order ? (int64_t)a.order[slot] : slot) : 0;

  // ---- the sample's set-up record (written by setup_kernel), read by part 0
  if (compute && part == 0) {
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    if (active) {
      r0 = a.rec[3 * s];
      r1 = a.rec[3 * s + 1];
      r2 = a.rec[3 * s + 2];
    }
    s_cf[0][row] = r0.x;
    s_cf[1][row] = r0.y;
    s_cf[2][row] = r0.z;
    s_cf[3][row] = r0.w;
    s_cf[4][row] = r1.x;
    s_cf[5][row] = r1.y;
    s_cf[6][row] = r1.z;
    s_cf[7][row] = r1.w;
    s_inv[row] = r2.x;
    s_kcut[row] = __float_as_int(r2.y);
  }
  if (tid == 0) {
    s_kmax = 0;
    s_bad = 0;
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bbar[b], 1);
      tc::mbar_init(&full[b], kACompute);
      tc::mbar_init(&mbar[b], 1);
      s_issued_b[b] = 0;
      s_issued_m[b] = 0;
    }
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc<512>(&s_tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  float cf[kNumBasis - 1];
#pragma unroll
  for (int j = 0; j < kNumBasis - 1; ++j) cf[j] = s_cf[j][row];
  const int32_t kcut = compute ? s_kcut[row] : 0;
  const float inv_s = compute ? s_inv[row] : 0.f;
  const bool valid = active && kcut > 0;
  if (compute && part == 0) atomicMax(&s_kmax, kcut);
  __syncthreads();
  const uint32_t tmem = s_tmem;
  const int32_t nkb_cta = (s_kmax + kTileBins - 1) / kTileBins;
  // blocks of pass p: the K-blocks that both the pass's templates and this CTA's samples reach
  auto pass_blocks = [&](int p) { return nkb_cta < a.nkb_pass[p] ? nkb_cta : a.nkb_pass[p]; };
  if (tid == 0) {
    int nb = 0;
    for (int p = 0; p < a.n_pass; ++p) nb += pass_blocks(p);
    s_nblk = nb;
  }
  // the basis records of the bins this CTA reaches, read by every compute thread in every
  // pass: staged once in shared memory when they fit (else read through L1)
  const int32_t n_rec4 = nkb_cta * (kTileBins / 2) * (kBinRecord / 4);
  const bool rec_smem = n_rec4 * 16 <= (int32_t)kRecSmem;
  float4* s_rec = reinterpret_cast<float4*>(sm + kAOffR);
  if (rec_smem) {
    const float4* src = reinterpret_cast<const float4*>(a.bins);
    for (int i = tid; i < n_rec4; i += kAThreads) s_rec[i] = __ldg(src + i);
  }
  __syncthreads();
  const int32_t nblk = s_nblk;

  unsigned char* sA = sm + kAOffA;
  unsigned char* sB = sm + kAOffB;
  bool bad = false;
  float best2 = -1.f;   // this thread's best |overlap|^2 and its slot p * 256 + i (compute threads)
  int32_t best_t = -1;

  if (!compute) {
    // ---- the MMA-issuer warp (one elected thread)
    if (lane == 0 && nblk > 0) {
      auto load_b = [&](int g, int p, int kb) {
        const int b = g & 1;
        const unsigned char* src = a.tiles + ((int64_t)p * a.g.n_kb + kb) * kBBlock;
        tc::mbar_expect_tx(&bbar[b], kBBlock);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          tc::bulk_g2s(sB + b * kBBlock + c * (kBBlock / 4), src + c * (kBBlock / 4), kBBlock / 4, &bbar[b]);
        ++s_issued_b[b];
      };
      int p = 0, kb = 0;
      while (p < a.n_pass && pass_blocks(p) == 0) ++p;
      load_b(0, p, 0);
      for (int g = 0; g < nblk; ++g) {
        const int b = g & 1;
        const uint32_t par = (uint32_t)((g >> 1) & 1);
        bool ok = tc::mbar_wait(&full[b], par) && tc::mbar_wait(&bbar[b], par);
        if (ok && s_bad) ok = false;
        if (!ok) {
          bad = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t a_base = tc::smem_addr(sA + b * kATile);
        const uint32_t b_base = tc::smem_addr(sB + b * kBBlock);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            tc::mma_f16(tmem + h * 2 * kTileTemplates, tc::desc_k_sw128(a_base + ks * 32),
                        tc::desc_k_sw128(b_base + h * kBHalf + ks * 32), kAIdesc, (kb > 0 || ks > 0) ? 1u : 0u);
        tc::commit(&mbar[b]);
        ++s_issued_m[b];
        // the next block: same pass or the next pass with blocks
        if (++kb >= pass_blocks(p)) {
          kb = 0;
          do {
            ++p;
          } while (p < a.n_pass && pass_blocks(p) == 0);
        }
        if (g + 1 < nblk) {
          // buffer b ^ 1 is free once the MMAs of block g - 1 completed
          ok = g < 1 || tc::mbar_wait(&mbar[b ^ 1], (uint32_t)(((g - 1) >> 1) & 1));
          if (!ok) {
            bad = true;
            break;
          }
          load_b(g + 1, p, kb);
        }
      }
      if (bad) {
        s_bad = 1;
        atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
      }
    }
    __syncwarp();
  } else {
    // ---- compute warps
    // TMEM columns [128 part, 128 part + 128): pass slots 64 part .. 64 part + 63
    const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(part * 128);
    // this thread's 64 overlaps of pass p against the running best, 16 at a time: the
    // chunk's maximum first, the slot only when it beats the best (the first slot visited
    // wins a tie)
    auto drain = [&](int p) {
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 32) {
        uint32_t r[32];
        tc::tmem_ld32(tbase + c0, r);
        float m2[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
          m2[i] = fmaf(re, re, im * im);
        }
        float cmax = m2[0];
#pragma unroll
        for (int i = 1; i < 16; ++i) cmax = fmaxf(cmax, m2[i]);
        if (cmax > best2) {
          int bi = 15;
#pragma unroll
          for (int i = 15; i >= 0; --i)
            if (m2[i] == cmax) bi = i;
          best2 = cmax;
          best_t = p * 2 * kTileTemplates + part * 64 + (c0 >> 1) + bi;
        }
      }
    };
    const float4* recs = rec_smem ? s_rec : reinterpret_cast<const float4*>(a.bins);
    unsigned char* rowA0 = sA + row * 128;
    int g = 0, last_p = -1;
    for (int p = 0; p < a.n_pass && !bad; ++p) {
      const int nb = pass_blocks(p);
      for (int kb = 0; kb < nb; ++kb, ++g) {
        const int b = g & 1;
        if (g >= 2) {
          // A[b] is free once the MMAs of block g - 2 completed
          const bool ok = tc::mbar_wait(&mbar[b], (uint32_t)(((g - 2) >> 1) & 1));
          if (__any_sync(0xffffffffu, !ok || s_bad)) {
            bad = true;
            break;
          }
        }
        unsigned char* rowA = rowA0 + b * kATile;
        // this thread's 8 bins of the block: 2 chunks of 16 bytes, 4 bins (8 FP16) each, the
        // values (Re a_k, Im a_k) of a_k = amp e^(-i 2 pi t_k)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int c = 2 * part + j;
          const int32_t k0 = kb * kTileBins + 4 * c;
          uint32_t wv[4];
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            const int32_t k = k0 + 2 * pr;
            const float4* rc = recs + (int64_t)(k >> 1) * (kBinRecord / 4);
            const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2], r3 = rc[3], r4 = rc[4];
            float2 t = __fmul2_rn(f2(cf[0]), make_float2(r0.x, r0.y));
            t = __ffma2_rn(f2(cf[1]), make_float2(r0.z, r0.w), t);
            t = __ffma2_rn(f2(cf[2]), make_float2(r1.x, r1.y), t);
            t = __ffma2_rn(f2(cf[3]), make_float2(r1.z, r1.w), t);
            t = __ffma2_rn(f2(cf[4]), make_float2(r2.x, r2.y), t);
            t = __ffma2_rn(f2(cf[5]), make_float2(r2.z, r2.w), t);
            t = __ffma2_rn(f2(cf[6]), make_float2(r3.x, r3.y), t);
            t = __ffma2_rn(f2(cf[7]), make_float2(r3.z, r3.w), t);
            t.x -= rintf(t.x);  // turns in [-1/2, 1/2]: the MUFU argument stays in [-pi, pi]
            t.y -= rintf(t.y);
            const float2 ang = __fmul2_rn(t, f2(-kTwoPiF));
            float2 sn, cs;
            __sincosf(ang.x, &sn.x, &cs.x);
            __sincosf(ang.y, &sn.y, &cs.y);
            float2 amp = __fmul2_rn(make_float2(r4.x, r4.y), f2(inv_s));
            if (k0 + 3 >= kcut) {  // the sample's ISCO cut falls in this chunk
              amp.x = k < kcut ? amp.x : 0.f;
              amp.y = k + 1 < kcut ? amp.y : 0.f;
            }
            const float2 re = __fmul2_rn(amp, cs), im = __fmul2_rn(amp, sn);
            const __half2 h0 = __floats2half2_rn(re.x, im.x), h1 = __floats2half2_rn(re.y, im.y);
            wv[2 * pr] = *reinterpret_cast<const uint32_t*>(&h0);
            wv[2 * pr + 1] = *reinterpret_cast<const uint32_t*>(&h1);
          }
          *reinterpret_cast<uint4*>(rowA + ((c ^ (row & 7)) << 4)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        if (kb == 0 && last_p >= 0) {
          // the pass that ended with block g - 1: read its overlaps before the MMAs of block g
          // start the accumulators afresh
          const bool ok = tc::mbar_wait(&mbar[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1));
          if (__any_sync(0xffffffffu, !ok || s_bad)) {
            bad = true;
            break;
          }
          tc::fence_after_sync();
          drain(last_p);
          tc::fence_before_sync();
        }
        tc::fence_proxy_async();
        tc::mbar_arrive(&full[b]);
      }
      if (nb > 0) last_p = p;
    }
    if (!bad && nblk > 0) {
      const bool ok = tc::mbar_wait(&mbar[(nblk - 1) & 1], (uint32_t)(((nblk - 1) >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok || s_bad)) {
        bad = true;
      } else {
        tc::fence_after_sync();
        drain(last_p);
        tc::fence_before_sync();
      }
    }
    if (bad) {
      s_bad = 1;
      atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
    }
  }
  // merge the four parts' bests of each sample (a tie goes to the lower template index)
  if (compute) {
    s_b2[part][row] = best2;
    s_bt[part][row] = best_t;
  }
  __syncthreads();
  if (compute && part == 0) {
#pragma unroll
    for (int o = 1; o < kParts; ++o) {
      const float o2 = s_b2[o][row];
      const int32_t ot = s_bt[o][row];
      if (ot >= 0 && (best_t < 0 || o2 > best2 || (o2 == best2 && ot < best_t))) {
        best2 = o2;
        best_t = ot;
      }
    }
    if (active) {
      const int32_t t = best_t >= 0 ? a.perm[best_t] : -1;
      const bool ok = valid && !s_bad && t >= 0;
      a.tile[s] = ok ? t : -1;
      if (a.match) a.match[s] = ok ? sqrtf(fmaxf(best2, 0.f)) : 0.f;
    }
  }
  if (tid == 0 && s_bad) {
    // let every copy and MMA issued land (bounded) before the CTA releases its memory
    for (int b = 0; b < 2; ++b) {
      if (s_issued_b[b] > 0) (void)tc::mbar_wait(&bbar[b], (uint32_t)((s_issued_b[b] - 1) & 1), 1000000000ull);
      if (s_issued_m[b] > 0) (void)tc::mbar_wait(&mbar[b], (uint32_t)((s_issued_m[b] - 1) & 1), 1000000000ull);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<512>(tmem);
}

// ---- stable counting sort of tile indices ---------------------------------------------
// hist[seg][j]: members of tile j in segment seg (kSortSegment consecutive samples)
__global__ void lists_hist_kernel(int64_t n, const int32_t* __restrict__ tile, int32_t T, int32_t* hist,
                                  int32_t* n_bad) {
  extern __shared__ int32_t h[];
  for (int32_t j = threadIdx.x; j < T; j += blockDim.x) h[j] = 0;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * kSortSegment, s1 = min(n, s0 + kSortSegment);
  int32_t bad = 0;
  for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    const int32_t j = tile[i];
    if (j >= 0 && j < T)
      atomicAdd(&h[j], 1);
    else
      ++bad;
  }
  if (bad) atomicAdd(n_bad, bad);
  __syncthreads();
  for (int32_t j = threadIdx.x; j < T; j += blockDim.x) hist[(int64_t)blockIdx.x * T + j] = h[j];
}

// per tile: exclusive scan of the segment counts (in place) and the total; then the tile
// offsets (one CTA)
__global__ void lists_scan_kernel(int32_t n_seg, int32_t T, int32_t* hist, int32_t* count, int32_t* offset) {
  for (int32_t j = threadIdx.x; j < T; j += blockDim.x) {
    int32_t run = 0;
    for (int32_t sg = 0; sg < n_seg; ++sg) {
      const int32_t v = hist[(int64_t)sg * T + j];
      hist[(int64_t)sg * T + j] = run;
      run += v;
    }
    count[j] = run;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int32_t j = 0; j < T; ++j) {
      offset[j] = run;
      run += count[j];
    }
  }
}

// one warp per segment, 32 samples per round in sample order: the rank of a sample among
// equal tiles of its round (lanes below it) plus the tile's count so far in the segment
__global__ void lists_scatter_kernel(int64_t n, const int32_t* __restrict__ tile, int32_t T,
                                     const int32_t* __restrict__ base, const int32_t* __restrict__ offset,
                                     int32_t* __restrict__ members) {
  extern __shared__ int32_t cnt[];
  const int lane = threadIdx.x;
  for (int32_t j = lane; j < T; j += 32) cnt[j] = 0;
  __syncwarp();
  const int64_t s0 = (int64_t)blockIdx.x * kSortSegment, s1 = min(n, s0 + kSortSegment);
  const int32_t* bs = base + (int64_t)blockIdx.x * T;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t r = s0; r < s1; r += 32) {
    const int64_t i = r + lane;
    int32_t j = (i < s1) ? tile[i] : -1;
    if (j >= T) j = -1;
    const unsigned same = __match_any_sync(0xffffffffu, j);
    const int rank = __popc(same & lt);
    if (j >= 0) members[offset[j] + bs[j] + cnt[j] + rank] = (int32_t)i;
    __syncwarp();
    if (j >= 0 && rank == 0) cnt[j] += __popc(same);
    __syncwarp();
  }
}

// ---- mixture over tiles (one CTA) ------------------------------------------------------
__global__ void mixture_kernel(int32_t T, const int32_t* __restrict__ count, const double* __restrict__ ll,
                               double* ll_copy, double* c, double* mix, int32_t* flag) {
  __shared__ double red[256];
  double m = -INFINITY;
  for (int32_t j = threadIdx.x; j < T; j += blockDim.x) {
    const double v = ll[j];
    ll_copy[j] = v;
    if (count[j] > 0 && v > m) m = v;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  m = red[0];
  if (threadIdx.x == 0) {
    // cumulative weights in tile order (the order of the definition)
    double s = 0.0;
    for (int32_t j = 0; j < T; ++j) {
      const double v = ll[j];
      if (count[j] > 0 && v > -INFINITY && v == v) s += (double)count[j] * exp(v - m);
      c[j] = s;
    }
    mix[0] = m;
    mix[1] = s;
    *flag = (m > -INFINITY && s > 0.0 && s < INFINITY) ? 0 : 1;
  }
}

// ---- mixture draws, one thread per draw ------------------------------------------------
__global__ void draw_kernel(TilingDrawArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint64_t g = a.ctr0 + (uint64_t)i;
  const Philox4 r = philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 3u, 0u, (uint32_t)a.seed,
                                  (uint32_t)(a.seed >> 32));
  const double total = a.mix[1];
  const uint64_t w0 = ((uint64_t)r.v[0] << 32) | r.v[1];
  const double target = (double)(w0 >> 11) * (1.0 / 9007199254740992.0) * total;
  int32_t lo = 0, hi = a.T - 1;  // first j with c_j > target
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (a.c[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  const int32_t j = lo;
  const uint64_t w1 = ((uint64_t)r.v[2] << 32) | r.v[3];
  const uint64_t k = __umul64hi(w1, (uint64_t)a.count[j]);
  const int32_t member = a.members[a.offset[j] + (int64_t)k];
  const double x = a.pool[member], q = a.pool[a.n_pool + member];
  double mc, qp;
  map_point(a.sp, x, q, mc, qp);
  if (a.coords) {
    a.coords[i] = x;
    a.coords[a.n + i] = q;
  }
  a.theta[i] = mc;
  a.theta[a.n + i] = qp;
  a.log_q[i] = a.log_prior + (a.ll[j] - a.mix[0] - log(total) + log((double)a.n_pool));
  a.log_p[i] = a.log_prior;
  if (a.pool_index) a.pool_index[i] = member;
}

}  // namespace

cudaError_t launch_tiling_waveforms(const TilingSpace& sp, const TilingGrid& g, int32_t n, const double* pts,
                                    double2* rows, double2* kmaj, int32_t ldk, int32_t col0, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  waveforms_kernel<<<n, 128, 0, s>>>(sp, g, n, pts, rows, kmaj, ldk, col0);
  return cudaGetLastError();
}

cudaError_t launch_tiling_absdots(int32_t na, const double2* A, int32_t nb, const double2* B, int32_t ldb, int32_t K,
                                  double* out, cudaStream_t s) {
  if (na <= 0 || nb <= 0) return cudaSuccess;
  dim3 grid((nb + kDotThreads - 1) / kDotThreads, (na + kDotRows - 1) / kDotRows);
  absdots_kernel<<<grid, kDotThreads, 0, s>>>(na, A, nb, B, ldb, K, out);
  return cudaGetLastError();
}

cudaError_t launch_tiling_pair_match(const TilingSpace& sp, const TilingGrid& g, int64_t n, const double* a,
                                     const double* b, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n * 32 + 255) / 256;
  pair_match_kernel<<<(unsigned)blocks, 256, 0, s>>>(sp, g, n, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_tiling_append(int32_t n, const int32_t* idx, const double2* src, int32_t K, double2* dst_rows,
                                 int32_t row0, double2* dst_kmaj, int32_t ldk, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  append_kernel<<<n, 128, 0, s>>>(n, idx, src, K, dst_rows, row0, dst_kmaj, ldk);
  return cudaGetLastError();
}

cudaError_t launch_tiling_bin_records(const TilingGrid& g, double wscale, float* out, cudaStream_t s) {
  const int32_t n = g.n_kb * (kTileBins / 2);
  bin_records_kernel<<<(n + 127) / 128, 128, 0, s>>>(g, wscale, out);
  return cudaGetLastError();
}

cudaError_t launch_tiling_template_tiles(const int32_t* perm, int32_t n_pass, const double2* rows, const TilingGrid& g,
                                         void* out, cudaStream_t s) {
  dim3 grid(g.n_kb, 2 * n_pass);
  template_tiles_kernel<<<grid, 256, 0, s>>>(perm, rows, g, static_cast<__half*>(out));
  return cudaGetLastError();
}

cudaError_t launch_tiling_setup(const TilingSpace& sp, const TilingGrid& g, int64_t n, const double* pts, float4* rec,
                                int32_t* kc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  setup_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sp, g, n, pts, rec, kc);
  return cudaGetLastError();
}

cudaError_t launch_tiling_assign(const AssignArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kASmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t blocks = (a.n + 127) / 128;
  assign_kernel<<<(unsigned)blocks, kAThreads, kASmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tiling_lists(int64_t n, const int32_t* tile, int32_t T, int32_t* hist, int32_t* count,
                                int32_t* offset, int32_t* n_bad, int32_t* members, cudaStream_t s) {
  const int64_t n_seg = (n + kSortSegment - 1) / kSortSegment;
  const size_t sh = sizeof(int32_t) * (size_t)T;
  if (sh > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(lists_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lists_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(n_bad, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  lists_hist_kernel<<<(unsigned)n_seg, 256, sh, s>>>(n, tile, T, hist, n_bad);
  lists_scan_kernel<<<1, 1024, 0, s>>>((int32_t)n_seg, T, hist, count, offset);
  lists_scatter_kernel<<<(unsigned)n_seg, 32, sh, s>>>(n, tile, T, hist, offset, members);
  return cudaGetLastError();
}

cudaError_t launch_tiling_mixture(int32_t T, const int32_t* count, const double* ll, double* ll_copy, double* c,
                                  double* mix, int32_t* flag, cudaStream_t s) {
  mixture_kernel<<<1, 256, 0, s>>>(T, count, ll, ll_copy, c, mix, flag);
  return cudaGetLastError();
}

cudaError_t launch_tiling_draw(const TilingDrawArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t blocks = (a.n + 255) / 256;
  draw_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mbis
