// k_tiling.cu -- kernels of the tiled proposal (Sec. II; App. A): FP64 waveforms and
// matches for template placement, the tensor-core tile assignment of prior samples, the
// stable per-tile member lists, the mixture over tiles and its draws.
//
// Waveforms are the TaylorF2 model of the likelihood (physics.cuh) at zero coalescence
// time and phase, whitened by one PSD and scaled to unit norm:
//   u_k = w_k e^(-i Psi(f_k)) / sqrt(sum_{k' < kcut} w_k'^2),  w_k = f_k^(-7/6) / sqrt(S_k),
// zero at and above the ISCO.  The match of two points is |sum_k conj(u_a,k) u_b,k|, the
// normalised overlap maximised over a constant phase.
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
  if (p >= g.n_kb * 8) return;
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

// Template operand: chunk c holds templates 128c .. 128c + 127 as 256 rows (template t:
// row 2t gives Re conj(a) b, row 2t + 1 Im conj(a) b against a sample row laid out as
// (Re a_k, Im a_k) pairs), one 16-bin K-block of 32 TF32 values per 128-byte row, 16-byte
// chunk c of row n at byte n * 128 + ((c ^ (n & 7)) << 4) (the 128-byte swizzle).
__global__ void template_tiles_kernel(int32_t T, const double2* __restrict__ rows, TilingGrid g, float* out) {
  const int32_t kb = blockIdx.x, chunk = blockIdx.y, n = threadIdx.x;
  const int32_t t = chunk * kTileTemplates + (n >> 1);
  const bool im = n & 1;
  float* tile = out + ((int64_t)chunk * g.n_kb + kb) * 8192;
  for (int kk = 0; kk < 16; ++kk) {
    const int32_t k = kb * 16 + kk;
    double2 v = make_double2(0.0, 0.0);
    if (t < T && k < g.K) v = rows[(int64_t)t * g.K + k];
    const float e[2] = {(float)(im ? v.y : v.x), (float)(im ? -v.x : v.y)};
    for (int h = 0; h < 2; ++h) {
      const int kidx = 2 * kk + h, c16 = kidx >> 2, pos = kidx & 3;
      tile[n * 32 + (((c16 ^ (n & 7)) << 2) | pos)] = tc::tf32_round(e[h]);
    }
  }
}

// ---- tile assignment on the tensor cores ------------------------------------------------
// The sample-by-template overlaps are a real contraction [samples x 2K] . [2K x 2T].  A CTA
// of 256 threads owns two tiles of 128 samples and visits the templates in passes of 128
// (one MMA column block of 256 per tile, TMEM columns [256 t, 256 t + 256)).  Per 16-bin
// K-block every thread writes its sample's 16 (Re, Im) pairs, rounded to TF32, into its
// row of a swizzled shared-memory tile; the block's template tile arrives by bulk copy;
// the last thread done issues 2 x 4 tcgen05.mma.kind::tf32 and commits to an mbarrier.
// After a pass's last K-block each thread reads its row's 128 complex overlaps back from
// TMEM (one block late, before the next pass's first MMA overwrites them) and keeps the
// running best.
constexpr int kAThreads = 256;
constexpr uint32_t kATile = 16384;                      // 128 rows x 128 bytes
constexpr uint32_t kBTile = 32768;                      // 256 rows x 128 bytes
constexpr uint32_t kAOffA = 0;                          // [2 buf][2 tile][kATile]
constexpr uint32_t kAOffB = kAOffA + 2 * 2 * kATile;    // [2 buf][kBTile]
constexpr uint32_t kASmem = kAOffB + 2 * kBTile + 1024;
constexpr uint32_t kAIdesc = tc::idesc_tf32(128, 2 * kTileTemplates);
constexpr float kTwoPiF = 6.28318530717958647692f;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__global__ void __launch_bounds__(kAThreads, 1) assign_kernel(AssignArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // bbar[b]: template tile of buffer b landed; full[b]: the 256 threads wrote A[b];
  // mbar[b]: the MMAs reading buffer b completed.
  __shared__ __align__(8) uint64_t bbar[2], full[2], mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_kmax, s_done[2];
  __shared__ int s_issued_b[2], s_issued_m[2];
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, tile = tid >> 7, row = tid & 127;
  const int64_t s = (int64_t)blockIdx.x * kAThreads + tid;
  const bool active = s < a.n;

  // ---- per-sample set-up (FP64), coefficients handed to FP32 in turns
  double x = 0.0, q = 1.0;
  if (active) {
    x = a.pts[s];
    q = a.pts[a.n + s];
  }
  const bool valid = active && in_space(a.sp, x, q);
  float cf[kNumBasis - 1];
  int32_t kcut = 0;
  float inv_s = 0.f;  // 1 / norm, with the table's weights scaled by 1 / wref
  if (valid) {
    const PointSetup ps = point_setup(a.sp, a.g, x, q);
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) cf[j] = (float)ps.pc.C[j];
    kcut = ps.kcut;
    inv_s = (float)(ps.inv_norm * a.g.wref);
  } else {
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) cf[j] = 0.f;
  }

  if (tid == 0) {
    s_kmax = 0;
    s_bad = 0;
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bbar[b], 1);
      tc::mbar_init(&full[b], kAThreads);
      tc::mbar_init(&mbar[b], 1);
      s_done[b] = 0;
      s_issued_b[b] = 0;
      s_issued_m[b] = 0;
    }
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc<512>(&s_tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  atomicMax(&s_kmax, kcut);
  __syncthreads();
  const uint32_t tmem = s_tmem;
  const int32_t nkb = (s_kmax + 15) / 16;  // K-blocks this CTA needs
  const int32_t nblk = nkb * a.n_chunk;    // blocks over all passes

  unsigned char* sA = sm + kAOffA;
  unsigned char* sB = sm + kAOffB;
  auto load_b = [&](int g) {
    const int b = g & 1;
    const int32_t pass = g / nkb, kb = g % nkb;
    const float* src = a.tiles + ((int64_t)pass * a.g.n_kb + kb) * 8192;
    tc::mbar_expect_tx(&bbar[b], kBTile);
    tc::bulk_g2s(sB + b * kBTile, src, kBTile / 2, &bbar[b]);
    tc::bulk_g2s(sB + b * kBTile + kBTile / 2, src + 4096, kBTile / 2, &bbar[b]);
    ++s_issued_b[b];
  };
  if (tid == 0 && nblk > 0) load_b(0);

  bool bad = false;
  float best2 = -1.f;
  int32_t best_t = -1;
  const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(tile * 2 * kTileTemplates);
  // this thread's 128 overlaps of pass `pass` against the running best (strictly greater:
  // the lowest template index wins a tie)
  auto drain = [&](int pass) {
#pragma unroll 1
    for (int c0 = 0; c0 < 2 * kTileTemplates; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tbase + c0, r);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
        const float m2 = fmaf(re, re, im * im);
        const int32_t t = pass * kTileTemplates + (c0 >> 1) + i;
        if (t < a.T && m2 > best2) {
          best2 = m2;
          best_t = t;
        }
      }
    }
  };

  const float4* recs = reinterpret_cast<const float4*>(a.bins);
  for (int32_t g = 0; g < nblk; ++g) {
    const int b = g & 1;
    const int32_t pass = g / nkb, kb = g % nkb;
    if (g >= 2) {
      // A[b] is free once the MMAs of block g - 2 completed
      const bool ok = tc::mbar_wait(&mbar[b], (uint32_t)(((g - 2) >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok || s_bad)) {
        bad = true;
        break;
      }
    }
    unsigned char* rowA = sA + (b * 2 + tile) * kATile + row * 128;
#pragma unroll 2
    for (int kk = 0; kk < 16; kk += 2) {
      const int32_t k = kb * 16 + kk;
      float4 hi = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < kcut) {
        const float4* rc = recs + (int64_t)(k >> 1) * (kBinRecord / 4);
        const float4 r0 = __ldg(rc), r1 = __ldg(rc + 1), r2 = __ldg(rc + 2), r3 = __ldg(rc + 3), r4 = __ldg(rc + 4);
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
        const float2 ang = __fmul2_rn(t, f2(kTwoPiF));
        float2 sn, cs;
        __sincosf(ang.x, &sn.x, &cs.x);
        __sincosf(ang.y, &sn.y, &cs.y);
        const float2 amp = __fmul2_rn(make_float2(r4.x, r4.y), f2(inv_s));
        const float2 re = __fmul2_rn(amp, cs), im = __fmul2_rn(amp, sn);  // u = amp e^(-i 2 pi t)
        hi = make_float4(tc::tf32_round(re.x), tc::tf32_round(-im.x), tc::tf32_round(re.y), tc::tf32_round(-im.y));
        if (k + 1 >= kcut) {
          hi.z = 0.f;
          hi.w = 0.f;
        }
      }
      const int chunk = (kk >> 1) ^ (row & 7);
      *reinterpret_cast<float4*>(rowA + (chunk << 4)) = hi;
    }
    if (kb == 0 && pass > 0) {
      // the pass that ended with block g - 1: read its overlaps before the MMAs of block g
      // start the accumulator afresh
      const bool ok = tc::mbar_wait(&mbar[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok || s_bad)) {
        bad = true;
        break;
      }
      tc::fence_after_sync();
      drain(pass - 1);
      tc::fence_before_sync();
    }
    tc::fence_proxy_async();
    tc::mbar_arrive(&full[b]);
    if (atomicAdd(&s_done[b], 1) == kAThreads - 1) {
      atomicExch(&s_done[b], 0);
      __threadfence_block();
      const uint32_t par = (uint32_t)((g >> 1) & 1);
      bool ok = tc::mbar_wait(&full[b], par) && tc::mbar_wait(&bbar[b], par);
      if (ok) {
        tc::fence_after_sync();
        const uint32_t a_base = tc::smem_addr(sA + b * 2 * kATile);
        const uint32_t b_base = tc::smem_addr(sB + b * kBTile);
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            tc::mma_tf32(tmem + t * 2 * kTileTemplates, tc::desc_k_sw128(a_base + t * kATile + ks * 32),
                         tc::desc_k_sw128(b_base + ks * 32), kAIdesc, (kb > 0 || ks > 0) ? 1u : 0u);
        tc::commit(&mbar[b]);
        ++s_issued_m[b];
        if (g + 1 < nblk) {
          // buffer b ^ 1 is free once the MMAs of block g - 1 completed
          ok = g < 1 || tc::mbar_wait(&mbar[b ^ 1], (uint32_t)(((g - 1) >> 1) & 1));
          if (ok) load_b(g + 1);
        }
      }
      if (!ok) {
        s_bad = 1;
        atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
      }
    }
  }
  if (!bad && nblk > 0) {
    const bool ok = tc::mbar_wait(&mbar[(nblk - 1) & 1], (uint32_t)(((nblk - 1) >> 1) & 1));
    if (__any_sync(0xffffffffu, !ok || s_bad)) {
      bad = true;
    } else {
      tc::fence_after_sync();
      drain(a.n_chunk - 1);
      tc::fence_before_sync();
    }
  }
  if (bad) {
    s_bad = 1;
    atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
  }
  __syncthreads();
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
  if (active) {
    const bool ok = valid && kcut > 0 && !bad && !s_bad && best_t >= 0;
    a.tile[s] = ok ? best_t : -1;
    if (a.match) a.match[s] = ok ? sqrtf(fmaxf(best2, 0.f)) : 0.f;
  }
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
  const int32_t n = g.n_kb * 8;
  bin_records_kernel<<<(n + 127) / 128, 128, 0, s>>>(g, wscale, out);
  return cudaGetLastError();
}

cudaError_t launch_tiling_template_tiles(int32_t T, const double2* rows, const TilingGrid& g, int32_t n_chunk,
                                         float* out, cudaStream_t s) {
  dim3 grid(g.n_kb, n_chunk);
  template_tiles_kernel<<<grid, 256, 0, s>>>(T, rows, g, out);
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
  const int64_t blocks = (a.n + kAThreads - 1) / kAThreads;
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
