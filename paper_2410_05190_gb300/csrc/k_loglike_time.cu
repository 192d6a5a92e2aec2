// k_loglike_time.cu -- fused likelihood with numeric time marginalisation (Sec. III) on the
// 5th-generation tensor cores.
//
//   a_k  = A sum_d P_d c_dk e^(-i (Psi_k + 2 pi f_k dt_d))          per sample, per bin
//   Re z_j = sum_k Re(a_k) cos(2 pi f_k tau_j) + Im(a_k) sin(2 pi f_k tau_j),  j = 0..127
//   ln L = ln[(1/128) sum_j exp(Re z_j - H/2)]
//
// The second line is a real contraction [samples x 2K] . [2K x 128 shifts].  A CTA owns a
// tile of 128 samples and runs two threads per sample (256 threads); two CTAs share an SM,
// so that one's per-sample set-up overlaps the other's blocks.  Per K-block of 16 bins:
//   * each thread computes its sample's a_k for one half of the block (8 bins), two bins at
//     a time in f32x2 (mixed-precision phase as in the folded kernel: anchors entered in
//     float-float when the event's phase terms allow it, FP64 otherwise; 32-bit fixed-point
//     turns positioned directly at the thread's first bin; FP32 remainder; MUFU sin/cos per
//     detector; each detector's delay and response argument as one 64-bit fixed-point turn
//     counter) and writes them, split into a TF32 head and an FP32 tail, into its sample's
//     row of a 128-byte-swizzled K-major shared-memory tile;
//   * the pre-swizzled twiddle tiles (head, tail) of the block arrive by cp.async.bulk, one
//     block ahead (the first warp to see a block's MMAs complete requests the next block's);
//   * the last warp done issues 3 x 4 tcgen05.mma.kind::tf32 of 128 shifts (M, the twiddle
//     tile) by 128 samples (N, the sample tile) -- head.head + head.tail +
//     tail.head for each 8-wide K step -- into a fresh TMEM accumulator, and commits to an
//     mbarrier.
// While the tensor core runs block kb the threads compute block kb + 1's rows; then they add
// block kb's accumulator into running sums kept in the other half of TMEM (FP32,
// round-to-nearest), which frees the accumulator for block kb + 1.  The per-sample set-up
// is split between the two threads of a sample (phase coefficients and cut on one, the
// detector responses and delays on the other) and exchanged through shared memory.  The A
// operand never touches global memory; after the last block the running sums go through
// shared memory (transposed) to the log-mean-exp.
#include "internal.h"
#include "marg.cuh"
#include "anchor.cuh"
#include "ffloat.cuh"
#include "setup_ff.cuh"
#include "tc.cuh"

namespace mbis {
namespace {

constexpr int kSamples = 128;           // samples per CTA: one tile of 128, one N = 128 MMA
constexpr int kTT = 2 * kSamples;       // two threads per sample
constexpr int kCtasPerSm = 2;
constexpr int kTilesPerCta = 1;
constexpr int kSegBins = kKBlockBins / 2;  // bins of a K-block per thread
constexpr uint32_t kTileBytes = 16384;  // 128 rows x 128 bytes
constexpr uint32_t kOffA = 0;           // [2 buf][2 head/tail][tile]
constexpr uint32_t kOffB = kOffA + 2 * kTilesPerCta * 2 * kTileBytes;  // [head/tail][tile], one buffer
constexpr uint32_t kOffC = kOffB + 2 * kTileBytes;                     // per-sample phase coefficients
constexpr int kPhaseFF = 2 * kNumBasis + 2;                            // 32-bit words per sample
constexpr uint32_t kSmemBytes = kOffC + (uint32_t)kPhaseFF * 4u * kSamples + 1024;
static_assert(kTimeShifts * (kSamples + 1) * 4 <= kOffC, "the final transpose fits the tiles' memory");
// D[shift][sample] = twiddle tile (M = 128 shifts) x sample tile (N = 128 samples, the CTA's
// tile)
constexpr uint32_t kIdesc = tc::idesc_tf32(kTimeShifts, kSamples);
// The tensor core aligns and truncates when it accumulates, which biases a long FP32
// accumulation toward zero by a fraction of an ulp per step.  Each K-block therefore
// accumulates in TMEM on its own: its two split corrections (head.tail, tail.head, ~2^-11
// smaller) first, into a fresh accumulator, then its four head.head products; the threads
// add the block's result into the running sums with round-to-nearest adds.
// TMEM (256 columns per CTA): [accumulator: columns 0..127 | running sums: 128..255],
// lanes = shifts.
constexpr uint32_t kTmemCols = 2 * kSamples;
constexpr uint32_t kRunCol = kSamples;
constexpr float kTwoPiF = 6.28318530717958647692f;
// Added to the 32-bit turn count: 256 rounds (rather than truncates) when its top 23 bits
// become a float mantissa f1 in [1, 2); 2^31 (half a turn) with the -3 pi in the remainder's
// constant puts the angle 2 pi f1 - 3 pi + ... in [-pi, pi), where the MUFU sine and cosine
// carry no mean phase error (over [0, 2 pi) they lag by ~1.7e-7 rad on average).
constexpr uint32_t kTurnOffset = 0x80000000u + 256u;

struct State {
  uint32_t acc, step;
  float c[kTimeRemDeg + 1];
  float w;
};

// Per-sample phase coefficients in shared memory, one column per sample (stride kSamples):
// float-float block entry: pf[j] = hi of C_j, pf[kNumBasis + j] = lo, then cst hi, lo;
// FP64 block entry: pd[j] = C_j, pd[kNumBasis] = cst.
__device__ __forceinline__ void enter_block(const AnchorBlock* __restrict__ plan, int blk, const double* pd,
                                            State& st) {
  const AnchorBlock& B = plan[blk];
  double x = pd[kNumBasis * kSamples], y = 0.0;
  float cf[kNumBasis - 1];
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    const double c = pd[j * kSamples];
    if (j < kNumBasis - 1) cf[j] = (float)c;
    x = fma(c, B.B[j], x);
    y = fma(c, B.dB[j], y);
  }
  const double w0 = (double)(B.k0 - B.kc);
  const double ph0 = fma(w0, y, x);
  const double f0 = ph0 - floor(ph0), fy = y - floor(y);
  const unsigned long long p0 = __double2ull_rn(f0 * 4294967296.0);
  const unsigned long long p1 = __double2ull_rn(fy * 4294967296.0);
  const double r0 = f0 - (double)p0 * 2.3283064365386963e-10;
  const double r1 = fy - (double)p1 * 2.3283064365386963e-10;
  st.acc = (uint32_t)p0 + kTurnOffset;
  st.step = (uint32_t)p1;
  remainder_coeffs<kTimeRemDeg>(B, [&](int j) { return cf[j]; }, st.c);
  st.c[0] += (float)(r0 - w0 * r1);
  st.c[1] += (float)r1;
#pragma unroll
  for (int m = 0; m <= kTimeRemDeg; ++m) st.c[m] *= kTwoPiF;
  st.c[0] -= 1.5f * kTwoPiF;
  st.w = (float)w0;
}

__device__ __forceinline__ void enter_block_ff(const AnchorBlock* __restrict__ plan, int blk, const float* pf,
                                               State& st) {
  const AnchorBlock& B = plan[blk];
  float xh = pf[2 * kNumBasis * kSamples], xl = pf[(2 * kNumBasis + 1) * kSamples], yh = 0.f, yl = 0.f;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    const float ch = pf[j * kSamples], cl = pf[(kNumBasis + j) * kSamples];
    const float4 q = __ldg(&B.Bq[j]);
    ff_mac(ch, cl, q.x, q.y, xh, xl);
    ff_mac(ch, cl, q.z, q.w, yh, yl);
  }
  two_sum(yh, yl, yh, yl);
  const float w0 = (float)(B.k0 - B.kc);
  ff_mac(w0, 0.f, yh, yl, xh, xl);  // phase at the block's first bin
  two_sum(xh, xl, xh, xl);
  float r0, r1;
  st.acc = ff_frac32(xh, xl, r0) + kTurnOffset;
  st.step = ff_frac32(yh, yl, r1);
  remainder_coeffs<kTimeRemDeg>(B, [&](int j) { return pf[j * kSamples]; }, st.c);
  st.c[0] += r0 - w0 * r1;
  st.c[1] += r1;
#pragma unroll
  for (int m = 0; m <= kTimeRemDeg; ++m) st.c[m] *= kTwoPiF;
  st.c[0] -= 1.5f * kTwoPiF;
  st.w = w0;
}

__device__ __forceinline__ float mantissa_turn(uint32_t a) { return __uint_as_float((a >> 9) | 0x3f800000u); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// kFF: anchor blocks entered in float-float (events whose phase terms stay below
// kFloatFloatMaxTurns), otherwise in FP64.  kRows: detector rows of the table (1 when the
// detectors are folded), a compile-time count so the detectors' chains interleave.
template <bool kFF, int kRows>
__global__ void __launch_bounds__(kTT, kCtasPerSm) loglike_mixed_time_kernel(LikeArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // bbar: the twiddle tiles of the current block landed; full[b]: every warp wrote its halves of the
  // rows of A[b] and added the previous block's accumulator into the running sums (one
  // arrival per warp); mbar[b]: the MMAs reading buffer b completed.  The last warp to arrive
  // for a block issues its MMAs from its first lane; the first warp to see them complete
  // requests the next block's twiddle tiles.  Decisions taken on a wait's outcome are
  // warp-uniform, since TMEM loads and stores are warp-collective.
  __shared__ __align__(8) uint64_t bbar, full[2], mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_kmax, s_done[2], s_bnext;
  __shared__ int s_issued_b, s_issued_m[2];
  __shared__ volatile int s_bad;
  __shared__ int32_t s_kcut[kSamples];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = tid / kSamples, si = tid % kSamples;
  const int tile = si >> 7, row = si & 127;
  constexpr int nrow = kRows;
  const int64_t slot = (int64_t)blockIdx.x * kSamples + si;
  const bool active = slot < a.n;
  const int64_t s = active && a.perm != nullptr ? (int64_t)a.perm[slot] : slot;

  // ---- per-sample set-up (FP64), shared by the sample's two threads
  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i)
    par[i] = (active && a.pos[i] >= 0) ? a.theta[(int64_t)a.pos[i] * a.n + s] : a.fixed[i];
  const bool valid = active && par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 &&
                     fabs(par[kChi2]) < 1.0 && par[kDl] > 0.0 && isfinite(par[kTc]) && isfinite(par[kPhic]) &&
                     isfinite(par[kRa]) && isfinite(par[kDec]) && isfinite(par[kPsi]) && isfinite(par[kIota]);
  // exchange area in the A tiles' memory (free until the first rows are written):
  // [detector][sample] |P_d|, delay counter offset and step, |P_d|^2
  float* x_pm = reinterpret_cast<float*>(sm + kOffA);
  uint64_t* x_off = reinterpret_cast<uint64_t*>(sm + kOffA + 4 * kMaxDet * kSamples);
  uint64_t* x_stp = x_off + kMaxDet * kSamples;
  double* x_p2 = reinterpret_cast<double*>(x_stp + kMaxDet * kSamples);
  double amp = 0.0;
  if (half == 0) {
    // phase coefficients, amplitude and cut (float-float set-up)
    SampleSetupFF ss;
#pragma unroll
    for (int j = 0; j < kNumBasis; ++j) ss.C[j] = FF{0.f, 0.f};
    ss.cst = FF{0.f, 0.f};
    ss.kcut = 0;
    ss.amp = 0.0;
    if (valid)
      ss = sample_setup_ff(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic], par[kDl], a.f_lo, a.df,
                           a.n_bins);
    const int32_t kcut = ss.kcut;
    amp = ss.amp;
    if constexpr (kFF) {
      float* pf = reinterpret_cast<float*>(sm + kOffC) + si;
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) {
        pf[j * kSamples] = ss.C[j].h;
        pf[(kNumBasis + j) * kSamples] = ss.C[j].l;
      }
      pf[2 * kNumBasis * kSamples] = ss.cst.h;
      pf[(2 * kNumBasis + 1) * kSamples] = ss.cst.l;
    } else {
      double* pd = reinterpret_cast<double*>(sm + kOffC) + si;
#pragma unroll
      for (int j = 0; j < kNumBasis; ++j) pd[j * kSamples] = ff_to_double(ss.C[j]);
      pd[kNumBasis * kSamples] = ff_to_double(ss.cst);
    }
    s_kcut[si] = kcut;
  } else if (!a.fold) {
    // Detector d enters as |P_d| c_dk e^{-i (Psi_k + 2 pi f_k dt_d - arg P_d)}: the argument
    // of the response and the delay share one 64-bit fixed-point turn counter (off, stp per
    // bin); the response argument enters the phase at FP32 accuracy.  Float-float throughout (~1e-14 relative; the FP64 pipe runs at a small fraction of
    // FP32): the angles' sines and cosines, the wave axes X, Y and the direction n once per
    // sample, then per detector F+ and Fx, |P|^2 (to FP64 for H), the response argument
    // (FP32 atan2) and the delay terms f_lo dt and df dt from the host's -f r / c.
    FF sp{0.f, 0.f}, cp{1.f, 0.f}, sd{0.f, 0.f}, cd{1.f, 0.f}, ss{0.f, 0.f}, cs{1.f, 0.f}, ci{1.f, 0.f};
    if (valid) {
      FF si;
      ff_sincos_any(par[kRa] - a.gmst, sp, cp);
      ff_sincos_any(par[kDec], sd, cd);
      ff_sincos_any(par[kPsi], ss, cs);
      ff_sincos_any(par[kIota], si, ci);
    }
    const FF cpsd = ff_mul(cp, sd), spsd = ff_mul(sp, sd);
    const FF X[3] = {ff_sub(ff_mul(sp, cs), ff_mul(ss, cpsd)), ff_neg(ff_add(ff_mul(cp, cs), ff_mul(ss, spsd))),
                     ff_mul(ss, cd)};
    const FF Y[3] = {ff_neg(ff_add(ff_mul(sp, ss), ff_mul(cs, cpsd))), ff_sub(ff_mul(cp, ss), ff_mul(cs, spsd)),
                     ff_mul(cs, cd)};
    const FF nv[3] = {ff_mul(cd, cp), ff_mul(cd, sp), sd};
    const FF cplus = ff_mul(FF{0.5f, 0.f}, ff_add_f(ff_mul(ci, ci), 1.0f));  // (1 + cos^2 iota) / 2
    auto dot = [&](const float (&r)[3][2], const FF (&v)[3]) {
      FF t = ff_mul(FF{r[0][0], r[0][1]}, v[0]);
      t = ff_add(t, ff_mul(FF{r[1][0], r[1][1]}, v[1]));
      return ff_add(t, ff_mul(FF{r[2][0], r[2][1]}, v[2]));
    };
#pragma unroll
    for (int d = 0; d < nrow; ++d) {
      float pm = 0.f;
      uint64_t off = 0, stp = 0;
      double p2 = 0.0;
      if (valid) {
        const FF xX = dot(a.det_xf[d], X), xY = dot(a.det_xf[d], Y), yX = dot(a.det_yf[d], X),
                 yY = dot(a.det_yf[d], Y);
        const FF fp = ff_mul(FF{0.5f, 0.f}, ff_add(ff_sub(ff_mul(xX, xX), ff_mul(xY, xY)),
                                                   ff_sub(ff_mul(yY, yY), ff_mul(yX, yX))));
        const FF fc = ff_sub(ff_mul(xX, xY), ff_mul(yX, yY));
        const FF p_re = ff_mul(fp, cplus), p_im = ff_neg(ff_mul(fc, ci));
        const FF q2 = ff_add(ff_mul(p_re, p_re), ff_mul(p_im, p_im));
        p2 = ff_to_double(q2);
        pm = sqrtf(q2.h);  // |P_d| enters in FP32
        constexpr FFConst kInv2Pi(1.0 / kTwoPi);
        const FF arg_turns = ff_mul(FF{atan2f(p_im.h, p_re.h), 0.f}, FF{kInv2Pi.h, kInv2Pi.l});
        off = ff_frac64(ff_sub(dot(a.det_offf[d], nv), arg_turns));
        stp = ff_frac64(dot(a.det_stpf[d], nv));
      }
      x_pm[d * kSamples + si] = pm;
      x_off[d * kSamples + si] = off;
      x_stp[d * kSamples + si] = stp;
      x_p2[d * kSamples + si] = p2;
    }
  }
  if (tid == 0) {
    s_kmax = 0;
    s_bad = 0;
    s_bnext = 0;
    s_issued_b = 0;
    tc::mbar_init(&bbar, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&full[b], kTT / 32);
      tc::mbar_init(&mbar[b], 1);
      s_done[b] = 0;
      s_issued_m[b] = 0;
    }
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc<kTmemCols>(&s_tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const int32_t kcut = s_kcut[si];
  float pmag[nrow];
  uint64_t off[nrow], stp[nrow];
  double H = 0.0;
  if (a.fold) {
#pragma unroll
    for (int d = 0; d < nrow; ++d) {
      pmag[d] = d == 0 ? 1.f : 0.f;
      off[d] = 0;
      stp[d] = 0;
    }
    if (half == 0 && valid) H = amp * amp * a.tfold[kcut];
  } else {
#pragma unroll
    for (int d = 0; d < nrow; ++d) {
      pmag[d] = x_pm[d * kSamples + si];
      off[d] = x_off[d * kSamples + si];
      stp[d] = x_stp[d * kSamples + si];
      if (half == 0 && valid) H += amp * amp * x_p2[d * kSamples + si] * a.tdet[(int64_t)d * (a.n_bins + 1) + kcut];
    }
  }
  if (half == 0) atomicMax(&s_kmax, kcut);
  __syncthreads();  // the exchange area is read before the first rows overwrite it
  const uint32_t tmem = s_tmem;
  const int32_t nkb = (s_kmax + kKBlockBins - 1) / kKBlockBins;
  const float* pf = reinterpret_cast<const float*>(sm + kOffC) + si;
  const double* pd = reinterpret_cast<const double*>(sm + kOffC) + si;

  unsigned char* sA = sm + kOffA;
  unsigned char* sB = sm + kOffB;
  const float* tiles = a.ttiles;
  // twiddle tiles of block kb into the buffer (one thread; the MMAs of block kb - 1 completed)
  auto load_b = [&](int kb) {
    tc::mbar_expect_tx(&bbar, 2 * kTileBytes);
    tc::bulk_g2s(sB, tiles + (int64_t)kb * 2 * 4096, kTileBytes, &bbar);
    tc::bulk_g2s(sB + kTileBytes, tiles + (int64_t)kb * 2 * 4096 + 4096, kTileBytes, &bbar);
    ++s_issued_b;
  };
  if (tid == 0 && nkb > 0) load_b(0);
  bool bad = false;
  // TMEM lanes are the shifts, columns the samples.  This warp adds the accumulator into the
  // running sums for its lane quarter (shifts 32 (warp % 4) + lane) over the 64 samples of
  // column group warp / 4, with round-to-nearest FP32 adds in block order.
  const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  auto drain = [&](bool first) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t r[16], q[16];
      if (first) {
        tc::tmem_ld16(tq + c0, r);
#pragma unroll
        for (int i = 0; i < 16; ++i) q[i] = 0u;
      } else {
        tc::tmem_ld16x2(tq + c0, r, tq + kRunCol + c0, q);  // block sums and running sums, one wait
      }
#pragma unroll
      for (int i = 0; i < 16; i += 2) {  // running sum + block sum, two lanes of f32x2
        const float2 u = __fadd2_rn(make_float2(__uint_as_float(q[i]), __uint_as_float(q[i + 1])),
                                    make_float2(__uint_as_float(r[i]), __uint_as_float(r[i + 1])));
        r[i] = __float_as_uint(u.x);
        r[i + 1] = __float_as_uint(u.y);
      }
      tc::tmem_st16(tq + kRunCol + c0, r);
    }
    tc::tmem_wait_st();
  };

  State st;
  st.acc = 0;
  st.step = 0;
  st.w = 0.f;
#pragma unroll
  for (int m = 0; m <= kTimeRemDeg; ++m) st.c[m] = 0.f;
  int blk = -1;
  int32_t blk_end = 0;
  uint32_t base[nrow], stepd[nrow], step2[nrow];
  float epsd[nrow];
#pragma unroll
  for (int d = 0; d < nrow; ++d) {
    base[d] = 0;
    stepd[d] = 0;
    step2[d] = 0;
    epsd[d] = 0.f;
  }
  // enter plan block blk at its first bin k0: the phase state, and per detector the 32-bit
  // turn counter at k0, its step per bin, and the fraction of a counter unit the step drops
  // per bin (as an FP32 slope)
  auto enter = [&](int32_t k0) {
    if constexpr (kFF)
      enter_block_ff(a.plan, blk, pf, st);
    else
      enter_block(a.plan, blk, pd, st);
    blk_end = a.plan[blk].k1;
#pragma unroll
    for (int d = 0; d < nrow; ++d) {
      const uint64_t od = off[d] + (uint64_t)(uint32_t)k0 * stp[d];
      base[d] = st.acc + (uint32_t)(od >> 32);
      stepd[d] = st.step + (uint32_t)(stp[d] >> 32);
      step2[d] = 2u * stepd[d];
      epsd[d] = (float)(uint32_t)stp[d] * (kTwoPiF * 5.421010862427522e-20f);  // 2 pi 2^-64
    }
  };
  int32_t blk_k0 = 0;
  for (int32_t kb = 0; kb < nkb; ++kb) {
    const int b = kb & 1;
    // this thread's half of the block: bins k_seg .. k_seg + 7 -> K values 16 half .. +15 of
    // its sample's row, 16-byte chunks 4 half .. 4 half + 3.  Buffer b is free: this thread
    // saw the MMAs of block kb - 2 complete before it drained them.
    const int32_t k_seg = kb * kKBlockBins + half * kSegBins;
    const float4* tab = reinterpret_cast<const float4*>(a.cdet32) + (int64_t)(k_seg >> 1);
    unsigned char* rowA = sA + ((b * 2) * kTilesPerCta + tile) * kTileBytes + row * 128;
    uint32_t cnt[nrow];
    float2 wv = f2(0.f), u2 = f2(0.f);  // bin - kc (remainder) and bin - k0 (counter slope)
#pragma unroll
    for (int d = 0; d < nrow; ++d) cnt[d] = 0;
    if (k_seg < kcut) {
      if (k_seg >= blk_end) {
        // the plan block holding the first bin (blocks may have begun in the other half)
        do {
          ++blk;
        } while (a.plan[blk].k1 <= k_seg);
        blk_k0 = a.plan[blk].k0;
        enter(blk_k0);
      }
      const uint32_t u = (uint32_t)(k_seg - blk_k0);
#pragma unroll
      for (int d = 0; d < nrow; ++d) cnt[d] = base[d] + u * stepd[d];
      wv = make_float2(st.w + (float)u, st.w + (float)u + 1.0f);
      u2 = make_float2((float)u, (float)u + 1.0f);
    }
#pragma unroll 1
    for (int kk = 0; kk < kSegBins; kk += 2) {
      const int32_t k = k_seg + kk;
      if (k < kcut && k == blk_end) {  // a plan block begins inside the half (plan blocks start on even bins)
        ++blk;
        blk_k0 = k;
        enter(k);
#pragma unroll
        for (int d = 0; d < nrow; ++d) cnt[d] = base[d];
        wv = make_float2(st.w, st.w + 1.0f);
        u2 = make_float2(0.f, 1.f);
      }
      float2 re = f2(0.f), imc = f2(0.f), ims = f2(0.f);  // im = imc - ims
      if (k < kcut) {
        float2 R = f2(st.c[kTimeRemDeg]);
#pragma unroll
        for (int m = kTimeRemDeg - 1; m >= 0; --m) R = __ffma2_rn(R, wv, f2(st.c[m]));
#pragma unroll
        for (int d = 0; d < nrow; ++d) {
          const float2 f1 = make_float2(mantissa_turn(cnt[d]), mantissa_turn(cnt[d] + stepd[d]));
          const float2 ang = __ffma2_rn(f1, f2(kTwoPiF), __ffma2_rn(f2(epsd[d]), u2, R));
          cnt[d] += step2[d];
          float2 sn, cs;
          __sincosf(ang.x, &sn.x, &cs.x);
          __sincosf(ang.y, &sn.y, &cs.y);
          const float4 c = __ldg(tab + (int64_t)d * (a.n_pad16 / 2) + (kk >> 1));  // re_k, re_k+1, im_k, im_k+1
          const float2 cx = make_float2(c.x, c.y), cy = make_float2(c.z, c.w);
          const float2 q = __fmul2_rn(f2(pmag[d]), cs), r = __fmul2_rn(f2(pmag[d]), sn);
          re = __ffma2_rn(cx, q, __ffma2_rn(cy, r, re));
          imc = __ffma2_rn(cy, q, imc);
          ims = __ffma2_rn(cx, r, ims);
        }
        if (k + 1 >= kcut) {  // odd cut: the second bin of the pair is beyond the ISCO
          re.y = 0.f;
          imc.y = 0.f;
          ims.y = 0.f;
        }
      }
      wv = __fadd2_rn(wv, f2(2.0f));
      u2 = __fadd2_rn(u2, f2(2.0f));
      const float2 im = __fadd2_rn(imc, make_float2(-ims.x, -ims.y));
      float4 hi, lo;
      // head and tail both rounded to TF32: the tensor core reads a TF32 operand by
      // truncating an FP32 one, which would bias the tails toward zero
      hi.x = tc::tf32_round(re.x); lo.x = tc::tf32_round(re.x - hi.x);
      hi.y = tc::tf32_round(im.x); lo.y = tc::tf32_round(im.x - hi.y);
      hi.z = tc::tf32_round(re.y); lo.z = tc::tf32_round(re.y - hi.z);
      hi.w = tc::tf32_round(im.y); lo.w = tc::tf32_round(im.y - hi.w);
      const int chunk = (half * (kSegBins / 2) + (kk >> 1)) ^ (row & 7);
      *reinterpret_cast<float4*>(rowA + (chunk << 4)) = hi;
      *reinterpret_cast<float4*>(rowA + kTilesPerCta * kTileBytes + (chunk << 4)) = lo;
    }
    tc::fence_proxy_async();
    if (kb >= 1) {
      // block kb - 1's accumulator into the running sums, once its MMAs completed (they ran
      // while this block's rows were computed); the accumulator is then free for block kb
      const bool ok = tc::mbar_wait(&mbar[(kb - 1) & 1], (uint32_t)(((kb - 1) >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok || s_bad)) {
        bad = true;
        break;
      }
      // the first warp to see them complete requests this block's twiddle tiles
      if (lane == 0 && atomicCAS(&s_bnext, kb - 1, kb) == kb - 1) load_b(kb);
      tc::fence_after_sync();
      drain(kb == 1);
    }
    tc::fence_before_sync();
    // one arrival per warp, once all its lanes wrote their rows and drained
    __syncwarp();
    int done = 0;
    if (lane == 0) {
      tc::mbar_arrive(&full[b]);
      done = atomicAdd(&s_done[b], 1);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (lane == 0 && done == kTT / 32 - 1) {
      // The last warp done with this block issues its MMAs.
      atomicExch(&s_done[b], 0);
      __threadfence_block();
      const uint32_t par = (uint32_t)((kb >> 1) & 1);
      bool ok = tc::mbar_wait(&full[b], par) && tc::mbar_wait(&bbar, (uint32_t)(kb & 1));
      if (ok) {
        tc::fence_after_sync();
        const uint32_t s_base = tc::smem_addr(sA + b * 2 * kTilesPerCta * kTileBytes);  // samples (N)
        const uint32_t w_base = tc::smem_addr(sB);                                      // twiddles (M)
        // the two split corrections (twiddle tail x sample head, twiddle head x sample tail)
        // first, started afresh, then the head x head products
#pragma unroll
        for (int term = 1; term <= 3; ++term)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const int tt = term % 3;  // 1: twiddle tail, 2: sample tail, 0: head x head
            const uint32_t ww = w_base + (tt == 1 ? kTileBytes : 0) + ks * 32;
            const uint32_t ss = s_base + (tt == 2 ? kTilesPerCta * kTileBytes : 0) + ks * 32;
            const bool fresh = term == 1 && ks == 0;
            tc::mma_tf32(tmem, tc::desc_k_sw128(ww), tc::desc_k_sw128(ss), kIdesc, fresh ? 0u : 1u);
          }
        tc::commit(&mbar[b]);
        ++s_issued_m[b];
      }
      if (!ok) {
        s_bad = 1;
        atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
      }
    }
  }
  if (!bad && nkb > 0) {
    // the last block's accumulator, once its MMAs (and so all) completed
    const bool ok = tc::mbar_wait(&mbar[(nkb - 1) & 1], (uint32_t)(((nkb - 1) >> 1) & 1));
    if (__any_sync(0xffffffffu, !ok || s_bad)) {
      bad = true;
    } else {
      tc::fence_after_sync();
      drain(nkb == 1);
    }
  }
  if (bad) {
    s_bad = 1;
    atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && s_bad) {
    // let every copy and MMA issued land (bounded) before the CTA releases its memory
    if (s_issued_b > 0) (void)tc::mbar_wait(&bbar, (uint32_t)((s_issued_b - 1) & 1), 1000000000ull);
    for (int b = 0; b < 2; ++b)
      if (s_issued_m[b] > 0) (void)tc::mbar_wait(&mbar[b], (uint32_t)((s_issued_m[b] - 1) & 1), 1000000000ull);
  }
  double ll = 0.0;
  if (nkb > 0 && !s_bad) {
    // every MMA and copy completed: the tiles' shared memory takes the running sums,
    // transposed to [shift][sample] (rows padded to 257 floats, conflict-free both ways)
    tc::fence_after_sync();
    constexpr int kT = kSamples + 1;
    float* zt = reinterpret_cast<float*>(sm);
    const int shift = 32 * (warp & 3) + (tid & 31), col0 = 64 * (warp >> 2);
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(tq + kRunCol + c0, r);
#pragma unroll
      for (int i = 0; i < 16; ++i) zt[shift * kT + col0 + c0 + i] = __uint_as_float(r[i]);
    }
    __syncthreads();
    if (half == 0) {
      float m = -INFINITY;
      for (int j = 0; j < kTimeShifts; ++j) m = fmaxf(m, zt[j * kT + si]);
      const double g = amp * a.cscale;  // Re z_j = g * running sum_j
      const float gf = (float)g;
      float sum = 0.f;
      for (int j = 0; j < kTimeShifts; ++j) sum += __expf(gf * (zt[j * kT + si] - m));
      // ln of a sum in [1, 128]: FP32 is exact to ~5e-7 absolute
      ll = g * (double)m + (double)logf(sum * (1.0f / kTimeShifts)) - 0.5 * H;
    }
  } else if (!s_bad) {
    ll = -0.5 * H;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<kTmemCols>(tmem);
  if (half == 0 && active) a.out[s] = (bad || s_bad) ? NAN : (valid ? ll : -INFINITY);
}

template <bool kFF, int kRows>
cudaError_t launch_time(const LikeArgs& a, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(loglike_mixed_time_kernel<kFF, kRows>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t blocks = (a.n + kSamples - 1) / kSamples;
  loglike_mixed_time_kernel<kFF, kRows><<<(unsigned)blocks, kTT, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

template <bool kFF>
cudaError_t launch_time_rows(const LikeArgs& a, cudaStream_t s) {
  switch (a.fold ? 1 : a.n_det) {
    case 1: return launch_time<kFF, 1>(a, s);
    case 2: return launch_time<kFF, 2>(a, s);
    case 3: return launch_time<kFF, 3>(a, s);
    default: return launch_time<kFF, 4>(a, s);
  }
}

}  // namespace

cudaError_t launch_loglike_mixed_time(const LikeArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return a.ff_phase ? launch_time_rows<true>(a, s) : launch_time_rows<false>(a, s);
}

}  // namespace mbis
