// k_loglike_mixed.cu -- fused waveform + projection + inner-product + marginalisation
// kernel in mixed precision (Eqs. 1-3 with the marginalised forms of Sec. III).  The
// waveform h(f) is never written to memory.
//
// One thread per proposal sample, 128 samples per CTA.  The folded data table C_k (FP32,
// detectors and their fixed responses folded in, stored as bin pairs
// (re_k, re_k+1, im_k, im_k+1)) streams through shared memory in chunks of 512 bins by TMA
// bulk copies (cp.async.bulk + mbarrier, two buffers); every thread of the CTA reads the
// same pair at the same time (one LDS.128 broadcast per two bins).
//
// Phase per bin (anchor blocks, see plan.cpp): at the start of a block each thread forms,
// in FP64 (or in float-float arithmetic when the event's phase terms stay below
// kFloatFloatMaxTurns), the linear phase X + (k - kc) Y, reduces it modulo one turn and keeps it as a
// 32-bit fixed-point turn count (exact wrap-around on integer add), and forms in FP32 the
// coefficients of the degree-5 remainder polynomial.  The FP64 rounding residuals of the
// fixed-point value and slope are folded into that polynomial.  Bins are taken in pairs
// with packed FP32x2 arithmetic: a 5-step Horner on both bins, the fixed-point -> float
// conversion through the mantissa, one FMA to radians, MUFU sine and cosine per bin, and
// a complex multiply-accumulate with C_k.  Per-chunk FP32 partial sums are accumulated in
// FP64.  The per-sample FP64 phase coefficients wait in shared memory between blocks so
// the loop keeps few registers (two CTAs more per SM).
#include "ffloat.cuh"
#include "internal.h"
#include "marg.cuh"
#include "tc.cuh"

namespace mbis {
namespace {

constexpr int kNbuf = 2;
constexpr float kTwoPiF = 6.28318530717958647692f;
// Added to the 32-bit turn count: 256 rounds (rather than truncates) when its top 23 bits
// become a float mantissa f1 in [1, 2); 2^31 (half a turn) with the -3 pi in the remainder's
// constant puts the angle 2 pi f1 - 3 pi + ... in [-pi, pi), where the MUFU sine and cosine
// carry no mean phase error (over [0, 2 pi) they lag by ~1.7e-7 rad on average).
constexpr uint32_t kTurnOffset = 0x80000000u + 256u;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

struct BlockState {
  uint32_t acc, step;
  float c[kFoldRemDeg + 1];
  float w;
};

// Enter anchor block blk: FP64 linear phase -> fixed point, FP32 remainder coefficients.
// pc / cf are this thread's coefficient columns in shared memory (stride T, the samples of
// a tile).
template <int T>
__device__ __forceinline__ void enter_block(const AnchorBlock* __restrict__ plan, int blk, const double* pc,
                                            const float* cf, BlockState& st) {
  const AnchorBlock& B = plan[blk];
  double x = pc[kNumBasis * T], y = 0.0;  // cst
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    const double Cj = pc[j * T];
    x = fma(Cj, B.B[j], x);
    y = fma(Cj, B.dB[j], y);
  }
  const double w0 = (double)(B.k0 - B.kc);
  const double ph0 = fma(w0, y, x);  // linear phase at the first bin of the block, turns
  const double f0 = ph0 - floor(ph0), fy = y - floor(y);
  const unsigned long long p0 = __double2ull_rn(f0 * 4294967296.0);
  const unsigned long long p1 = __double2ull_rn(fy * 4294967296.0);
  const double r0 = f0 - (double)p0 * 2.3283064365386963e-10;  // rounding residuals, turns
  const double r1 = fy - (double)p1 * 2.3283064365386963e-10;
  st.acc = (uint32_t)p0 + kTurnOffset;
  st.step = (uint32_t)p1;
#pragma unroll
  for (int m = 0; m <= kFoldRemDeg; ++m) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) s = fmaf(cf[j * T], B.E[j][m], s);
    st.c[m] = s;
  }
  st.c[0] += (float)(r0 - w0 * r1);
  st.c[1] += (float)r1;
  // angle = 2 pi (acc / 2^32) + 2 pi R = 2 pi f1 + (2 pi R - 3 pi), f1 = 1 + (acc + 2^31) / 2^32
#pragma unroll
  for (int m = 0; m <= kFoldRemDeg; ++m) st.c[m] *= kTwoPiF;
  st.c[0] -= 1.5f * kTwoPiF;
  st.w = (float)w0;
}

// The same entry in float-float arithmetic (events whose phase terms stay below
// kFloatFloatMaxTurns; no FP64).  pf is this thread's column (stride T): C_j hi at row j,
// cst hi at row kNumBasis, C_j lo at row kNumBasis + 1 + j, cst lo at the last.
template <int T>
__device__ __forceinline__ void enter_block_ff(const AnchorBlock* __restrict__ plan, int blk, const float* pf,
                                               BlockState& st) {
  constexpr int S = T, L = kNumBasis + 1;
  const AnchorBlock& B = plan[blk];
  float xh = pf[kNumBasis * S], xl = pf[(L + kNumBasis) * S], yh = 0.f, yl = 0.f;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    const float ch = pf[j * S], cl = pf[(L + j) * S];
    ff_mac(ch, cl, B.Bq[j].x, B.Bq[j].y, xh, xl);
    ff_mac(ch, cl, B.Bq[j].z, B.Bq[j].w, yh, yl);
  }
  two_sum(yh, yl, yh, yl);
  const float w0 = (float)(B.k0 - B.kc);
  ff_mac(w0, 0.f, yh, yl, xh, xl);  // linear phase at the first bin of the block, turns
  two_sum(xh, xl, xh, xl);
  float r0, r1;
  st.acc = ff_frac32(xh, xl, r0) + kTurnOffset;
  st.step = ff_frac32(yh, yl, r1);
#pragma unroll
  for (int m = 0; m <= kFoldRemDeg; ++m) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) s = fmaf(pf[j * S], B.E[j][m], s);
    st.c[m] = s;
  }
  st.c[0] += r0 - w0 * r1;
  st.c[1] += r1;
#pragma unroll
  for (int m = 0; m <= kFoldRemDeg; ++m) st.c[m] *= kTwoPiF;
  st.c[0] -= 1.5f * kTwoPiF;
  st.w = w0;
}

__device__ __forceinline__ float mantissa_turn(uint32_t a) { return __uint_as_float((a >> 9) | 0x3f800000u); }

// Shared memory of one CTA of T threads (declared once per kernel, so the persistent
// launch's two instantiations of fold_tile share it).
template <int T>
struct FoldSmem {
  __align__(128) float4 sC[kNbuf][kChunk / 2];
  __align__(8) uint64_t bar[kNbuf];
  double sPC[(kNumBasis + 1) * T];  // C_j and cst per thread (float pairs when kFF)
  float sCF[(kNumBasis - 1) * T];   // FP32 copies of C_0..C_7 (FP64 entry only)
  int s_kmax;
};

// log L of one sample from its overlap sums (in units of cscale / A) and its set-up:
// the marginalisations of Sec. III.  Shared by the kernel and the split launch's epilogue.
__device__ __forceinline__ double fold_loglike(const LikeArgs& a, double A, int32_t kcut, double Zr, double Zi) {
  const double zr = A * a.cscale * Zr, zi = A * a.cscale * Zi;
  const double H = A * A * a.tfold[kcut];
  if (a.marg == 0) return zr - 0.5 * H;
  if (a.marg == MBIS_MARG_PHASE) return log_i0(hypot(zr, zi)) - 0.5 * H;
  return log_distance_marginal_mixed(hypot(zr, zi), H, a.dist, a.glf);
}

// One tile of T samples of one event (one per thread).  `first` is false when the CTA has
// already run a tile (persistent launch): the mbarriers are then invalidated and initialised
// afresh.  piece / split: this CTA sums the parts [n_parts piece / split, n_parts (piece + 1)
// / split) of the tile's bins; with split > 1 it writes their sums for the epilogue kernel.
// A sample's arithmetic does not depend on T or on its tile-mates.
template <bool kFF, int T>
__device__ __forceinline__ void fold_tile(const LikeArgs& a, int64_t tile, bool first, FoldSmem<T>& sm, int piece = 0,
                                          int split = 1) {
  float4 (&sC)[kNbuf][kChunk / 2] = sm.sC;
  uint64_t* bar = sm.bar;
  double* sPC = sm.sPC;
  float* sCF = sm.sCF;
  int& s_kmax = sm.s_kmax;
  const int tid = threadIdx.x;
  const int64_t slot = tile * T + tid;
  const bool active = slot < a.n;
  const int64_t s = active && a.perm != nullptr ? (int64_t)a.perm[slot] : slot;

  // ---- per-sample set-up (FP64)
  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i) par[i] = (active && a.pos[i] >= 0) ? a.theta[(int64_t)a.pos[i] * a.n + s] : a.fixed[i];
  if (a.marg & MBIS_MARG_PHASE) par[kPhic] = 0.0;
  if (a.marg & MBIS_MARG_DISTANCE) par[kDl] = 1.0;
  const bool valid = active && par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 &&
                     fabs(par[kChi2]) < 1.0 && par[kDl] > 0.0 && isfinite(par[kTc]) && isfinite(par[kPhic]);
  int32_t kcut = 0;
  double A = 0.0;
  {
    PhaseCoeffs pc;
    if (valid) {
      const SampleSetup ss = sample_setup(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic], par[kDl],
                                          a.f_lo, a.df, a.n_bins);
      pc = ss.pc;
      kcut = ss.kcut;
      A = ss.amp;
    } else {
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) pc.C[j] = 0.0;
      pc.cst = 0.0;
    }
    if constexpr (kFF) {
      float* pf = reinterpret_cast<float*>(sPC) + tid;
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) {
        const float h = (float)pc.C[j];
        pf[j * T] = h;
        pf[(kNumBasis + 1 + j) * T] = (float)(pc.C[j] - (double)h);
      }
      const float h = (float)pc.cst;
      pf[kNumBasis * T] = h;
      pf[(2 * kNumBasis + 1) * T] = (float)(pc.cst - (double)h);
    } else {
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) sPC[j * T + tid] = pc.C[j];
      sPC[kNumBasis * T + tid] = pc.cst;
#pragma unroll
      for (int j = 0; j < kNumBasis - 1; ++j) sCF[j * T + tid] = (float)pc.C[j];
    }
  }
  const double* my_pc = sPC + tid;
  const float* my_cf = sCF + tid;
  const float* my_pf = reinterpret_cast<const float*>(sPC) + tid;

  if (tid == 0) {
    s_kmax = 0;
    if (!first)
      for (int b = 0; b < kNbuf; ++b) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(&bar[b])) : "memory");
    for (int b = 0; b < kNbuf; ++b) tc::mbar_init(&bar[b], 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  atomicMax(&s_kmax, kcut);
  __syncthreads();
  const int32_t kmax = s_kmax;
  const int32_t nch = (kmax + kChunk - 1) / kChunk;
  const int32_t n_parts = (a.n_bins + kPartBins - 1) / kPartBins;
  const int32_t part_lo = (int32_t)((int64_t)n_parts * piece / split);
  const int32_t part_hi = (int32_t)((int64_t)n_parts * (piece + 1) / split);
  const int32_t ch_lo = min(part_lo * kPartChunks, nch), ch_hi = min(part_hi * kPartChunks, nch);
  constexpr uint32_t kBytes = kChunk * sizeof(float2);
  int issued[kNbuf] = {};  // copies issued per buffer (thread 0)
  if (tid == 0) {
    for (int b = 0; b < kNbuf && ch_lo + b < ch_hi; ++b) {
      tc::mbar_expect_tx(&bar[b], kBytes);
      tc::bulk_g2s(sC[b], a.cfold32 + (int64_t)(ch_lo + b) * (kChunk / 2), kBytes, &bar[b]);
      ++issued[b];
    }
  }

  // ---- sweep over frequency
  FFSum Zr, Zi;  // the part's chunk sums (FP32), added without FP64 arithmetic
  double Zr_tot = 0.0, Zi_tot = 0.0;  // the parts, in order
  int32_t part = part_lo;
  BlockState st;
  int32_t blk_end = 0;
  int blk = -1;
  if (ch_lo > 0) {
    // start inside the grid: the anchor block that holds the range's first bin (entered,
    // then advanced to that bin below)
    const int32_t k0 = ch_lo * kChunk;
    int lo = 0, hi = a.n_blocks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.plan[mid].k0 <= k0)
        lo = mid;
      else
        hi = mid - 1;
    }
    blk = lo - 1;
    blk_end = k0;
  }
  bool timed_out = false;
  for (int32_t ch = ch_lo; ch < ch_hi; ++ch) {
    const int b = (ch - ch_lo) % kNbuf;
    const bool got = tc::mbar_wait(&bar[b], (uint32_t)(((ch - ch_lo) / kNbuf) & 1));
    if (__syncthreads_or(!got)) {
      timed_out = true;
      break;
    }
    const float4* __restrict__ cb = sC[b];
    const int32_t kb = ch * kChunk, ke = min(kb + kChunk, kmax);
    float2 zr = f2(0.f), zi = f2(0.f), zn = f2(0.f);  // zn accumulates re(C) sin, subtracted at the end
    int32_t k = kb;
    while (k < ke) {
      if (k == blk_end) {
        ++blk;
        if (k < kcut) {
          if constexpr (kFF)
            enter_block_ff<T>(a.plan, blk, my_pf, st);
          else
            enter_block<T>(a.plan, blk, my_pc, my_cf, st);
          // a range that starts inside the block: the state at bin k, exactly as a sweep
          // from the block's first bin reaches it (integer turn counter, integer offset)
          const int32_t adv = k - a.plan[blk].k0;
          st.acc += (uint32_t)adv * st.step;
          st.w += (float)adv;
        }
        blk_end = a.plan[blk].k1;
      }
      const int32_t seg_end = min(ke, blk_end);
      const int32_t my_end = min(seg_end, kcut);
      if (k < my_end) {
        float2 cr[kFoldRemDeg + 1];  // remainder coefficients, both lanes
#pragma unroll
        for (int m = 0; m <= kFoldRemDeg; ++m) cr[m] = f2(st.c[m]);
        const float2 two = f2(2.0f), twopi = f2(kTwoPiF);
        const uint32_t step = st.step, step2 = 2u * st.step;
        uint32_t acc = st.acc;
        float2 w = make_float2(st.w, st.w + 1.0f);
        const int32_t npair = (my_end - k) >> 1;
        const float4* cp = cb + ((k - kb) >> 1);
#pragma unroll 1
        for (int32_t p = 0; p < npair; ++p) {
          float2 R = cr[kFoldRemDeg];
#pragma unroll
          for (int m = kFoldRemDeg - 1; m >= 0; --m) R = __ffma2_rn(R, w, cr[m]);
          const float2 f1 = make_float2(mantissa_turn(acc), mantissa_turn(acc + step));
          const float2 ang = __ffma2_rn(f1, twopi, R);
          float2 sn, cs;
          __sincosf(ang.x, &sn.x, &cs.x);
          __sincosf(ang.y, &sn.y, &cs.y);
          const float4 c = cp[p];
          const float2 cre = make_float2(c.x, c.y), cim = make_float2(c.z, c.w);
          zr = __ffma2_rn(cre, cs, __ffma2_rn(cim, sn, zr));
          zi = __ffma2_rn(cim, cs, zi);
          zn = __ffma2_rn(cre, sn, zn);
          acc += step2;
          w = __fadd2_rn(w, two);
        }
        int32_t kk = k + 2 * npair;
        if (kk < my_end) {  // one bin left (odd cut): the even half of the pair
          float R = st.c[kFoldRemDeg];
#pragma unroll
          for (int m = kFoldRemDeg - 1; m >= 0; --m) R = fmaf(R, w.x, st.c[m]);
          const float ang = fmaf(mantissa_turn(acc), kTwoPiF, R);
          float sn, cs;
          __sincosf(ang, &sn, &cs);
          const float4 c = cp[npair];
          zr.x = fmaf(c.x, cs, fmaf(c.z, sn, zr.x));
          zi.x = fmaf(c.z, cs, zi.x);
          zn.x = fmaf(c.x, sn, zn.x);
          acc += step;
          w.x += 1.0f;
          ++kk;
        }
        st.acc = acc;
        st.w = w.x;
      }
      k = seg_end;
    }
    Zr.add(zr.x);
    Zr.add(zr.y);
    Zi.add(zi.x);
    Zi.add(zi.y);
    Zi.add(-zn.x);
    Zi.add(-zn.y);
    if ((ch + 1) % kPartChunks == 0 || ch + 1 == ch_hi) {
      // the part ends here
      if (split > 1) {
        if (active) a.zpart[(int64_t)part * a.n + s] = make_double2(Zr.value(), Zi.value());
      } else {
        Zr_tot += Zr.value();
        Zi_tot += Zi.value();
      }
      Zr = FFSum{};
      Zi = FFSum{};
      ++part;
    }
    __syncthreads();  // every thread is done with buffer b
    if (tid == 0 && ch + kNbuf < ch_hi) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_expect_tx(&bar[b], kBytes);
      tc::bulk_g2s(sC[b], a.cfold32 + (int64_t)(ch + kNbuf) * (kChunk / 2), kBytes, &bar[b]);
      ++issued[b];
    }
  }
  if (timed_out) {
    if (tid == 0) {
      atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
      // let the last copy issued into each buffer land (bounded) before the CTA's shared
      // memory is released
      for (int bb = 0; bb < kNbuf; ++bb)
        if (issued[bb] > 0) (void)tc::mbar_wait(&bar[bb], (uint32_t)((issued[bb] - 1) & 1));
    }
    if (active) {
      if (split > 1) {
        for (int32_t q = part_lo; q < part_hi; ++q) a.zpart[(int64_t)q * a.n + s] = make_double2(NAN, NAN);
        if (piece == 0) a.amp_out[s] = NAN;
      } else {
        a.out[s] = NAN;
      }
    }
    return;
  }
  if (!active) return;
  if (split > 1) {
    // parts of this piece beyond the tile's last live bin are empty; the first piece passes on
    // the sample's set-up
    for (; part < part_hi; ++part) a.zpart[(int64_t)part * a.n + s] = make_double2(0.0, 0.0);
    if (piece == 0) {
      a.amp_out[s] = valid ? A : -1.0;
      a.kcut_out[s] = kcut;
    }
    return;
  }
  if (!valid) {
    a.out[s] = -INFINITY;
    return;
  }
  // ---- marginalisation (Sec. III)
  a.out[s] = fold_loglike(a, A, kcut, Zr_tot, Zi_tot);
}

// The split launch's epilogue: a sample's parts in order, then its log L.
__global__ void fold_epilogue_kernel(LikeArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const double A = a.amp_out[s];
  if (!(A >= 0.0)) {
    a.out[s] = A < 0.0 ? -INFINITY : NAN;
    return;
  }
  const int32_t n_parts = (a.n_bins + kPartBins - 1) / kPartBins;
  double Zr = 0.0, Zi = 0.0;
  for (int32_t q = 0; q < n_parts; ++q) {
    const double2 z = a.zpart[(int64_t)q * a.n + s];
    Zr += z.x;
    Zi += z.y;
  }
  a.out[s] = fold_loglike(a, A, a.kcut_out[s], Zr, Zi);
}

template <bool kFF>
__global__ void __launch_bounds__(kMixedThreads, 8) loglike_mixed_fold_kernel(LikeArgs a) {
  __shared__ FoldSmem<kMixedThreads> sm;
  const int split = a.split > 1 ? a.split : 1;
  fold_tile<kFF, kMixedThreads>(a, blockIdx.x / split, true, sm, (int)(blockIdx.x % split), split);
}

// Persistent launch over the tiles of many events: each CTA takes (event, tile) items from a
// device counter until the list is exhausted.  The host orders the list longest first, so
// uneven events (2k-128k bins, 2^14-2^20 samples) balance across the SMs.  One launch
// takes the events of one block-entry arithmetic (kFF), so each keeps its own registers.
// Tiles of T samples with at most C CTAs per SM (the autotuner picks among (64, 14),
// (128, 7) and (256, 3)): 72-85 registers hold the persistent loop's state without the
// spills that a 64-register bound caused (6% faster on the uneven batch at T = 128).
template <bool kFF, int T, int C>
__global__ void __launch_bounds__(T, C) loglike_mixed_batch_kernel(const LikeArgs* __restrict__ args,
                                                                   const BatchItem* __restrict__ items, int32_t n_items,
                                                                   int32_t* next) {
  __shared__ int s_item;
  __shared__ FoldSmem<T> sm;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const BatchItem item = items[it];
    fold_tile<kFF, T>(args[item.ev], item.tile, first, sm);
    first = false;
    __syncthreads();
  }
}

}  // namespace

int32_t batch_ctas_per_sm(int32_t tile) {
  switch (tile) {
    case 64: return 14;
    case 256: return 3;
    default: return kBatchCtasPerSm;
  }
}

cudaError_t launch_loglike_mixed_batch(const LikeArgs* args, const BatchItem* items, int32_t n_items, int32_t* next,
                                      int32_t grid, bool ff, int32_t tile, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  switch (tile) {
    case 64:
      if (ff)
        loglike_mixed_batch_kernel<true, 64, 14><<<grid, 64, 0, s>>>(args, items, n_items, next);
      else
        loglike_mixed_batch_kernel<false, 64, 14><<<grid, 64, 0, s>>>(args, items, n_items, next);
      break;
    case 256:
      if (ff)
        loglike_mixed_batch_kernel<true, 256, 3><<<grid, 256, 0, s>>>(args, items, n_items, next);
      else
        loglike_mixed_batch_kernel<false, 256, 3><<<grid, 256, 0, s>>>(args, items, n_items, next);
      break;
    case kMixedThreads:
      if (ff)
        loglike_mixed_batch_kernel<true, kMixedThreads, kBatchCtasPerSm><<<grid, kMixedThreads, 0, s>>>(args, items,
                                                                                                      n_items, next);
      else
        loglike_mixed_batch_kernel<false, kMixedThreads, kBatchCtasPerSm><<<grid, kMixedThreads, 0, s>>>(args, items,
                                                                                                       n_items, next);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_loglike_mixed(const LikeArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int split = a.split > 1 ? a.split : 1;
  const int64_t blocks = (a.n + kMixedThreads - 1) / kMixedThreads * split;
  if (a.ff_phase)
    loglike_mixed_fold_kernel<true><<<(unsigned)blocks, kMixedThreads, 0, s>>>(a);
  else
    loglike_mixed_fold_kernel<false><<<(unsigned)blocks, kMixedThreads, 0, s>>>(a);
  if (split > 1) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_epilogue_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace mbis
