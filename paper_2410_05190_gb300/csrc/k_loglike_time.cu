// k_loglike_time.cu -- fused likelihood with numeric time marginalisation (Sec. III) on the
// 5th-generation tensor cores.
//
//   a_k  = A sum_d P_d c_dk e^(-i (Psi_k + 2 pi f_k dt_d))          per sample, per bin
//   Re z_j = sum_k Re(a_k) cos(2 pi f_k tau_j) + Im(a_k) sin(2 pi f_k tau_j),  j = 0..127
//   ln L = ln[(1/128) sum_j exp(Re z_j - H/2)]
//
// The second line is a real contraction [samples x 2K] . [2K x 128 shifts].  A CTA of 256
// threads owns two tiles of 128 samples.  Per K-block of 16 bins:
//   * every thread computes its sample's a_k for the 16 bins (mixed-precision phase as in
//     the folded kernel: FP64 anchors, 32-bit fixed-point turns, FP32 remainder, MUFU
//     sin/cos per detector; detector delays as 64-bit fixed-point turn counters) and writes
//     them, split into a TF32 head and an FP32 tail, into its row of a 128-byte-swizzled
//     K-major shared-memory tile;
//   * the pre-swizzled twiddle tiles (head, tail) of the block arrive by cp.async.bulk;
//   * one thread issues 3 x 4 x 2 tcgen05.mma.kind::tf32 (head.head + head.tail + tail.head
//     for each 8-wide K step and both tiles) accumulating in TMEM and commits to an mbarrier
//     that frees the double buffer two blocks later.
// The A operand never touches global memory.  Every few blocks each thread reads its own
// row (its 128 shifts) back from TMEM into FP32 registers; after the last block it applies
// the log-mean-exp.
#include "internal.h"
#include "marg.cuh"
#include "tc.cuh"

namespace mbis {
namespace {

constexpr int kTT = 256;
constexpr int kTilesPerCta = 2;
constexpr uint32_t kTileBytes = 16384;  // 128 rows x 128 bytes
constexpr uint32_t kOffA = 0;           // [2 buf][2 tile][2 head/tail][tile]
constexpr uint32_t kOffB = kOffA + 2 * kTilesPerCta * 2 * kTileBytes;  // [2 buf][2 head/tail][tile]
constexpr uint32_t kOffC = kOffB + 2 * 2 * kTileBytes;                 // [2 buf][kMaxDet][16] float2
constexpr uint32_t kSmemBytes = kOffC + 2 * kMaxDet * kKBlockBins * 8 + 1024;
constexpr uint32_t kIdesc = tc::idesc_tf32(128, kTimeShifts);
// The tensor core aligns and truncates when it accumulates, which biases a long FP32
// accumulation toward zero by a fraction of an ulp per step.  Each accumulator therefore
// takes at most kSegBlocks K-blocks (4 MMA steps each for the main term) before it is drained
// into FP32 registers with round-to-nearest adds; the split corrections, ~2^-11 smaller,
// accumulate separately.  TMEM: per tile [main 128 | correction 128] columns.
constexpr int kSegBlocks = 4;
constexpr float kTwoPiF = 6.28318530717958647692f;

struct State {
  uint32_t acc, step;
  float c[kRemDeg + 1];
  float w;
};

__device__ __forceinline__ void enter_block(const AnchorBlock* __restrict__ plan, int blk, const PhaseCoeffs& pc,
                                            const float* cf, State& st) {
  const AnchorBlock& B = plan[blk];
  double x = pc.cst, y = 0.0;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    x = fma(pc.C[j], B.B[j], x);
    y = fma(pc.C[j], B.dB[j], y);
  }
  const double w0 = (double)(B.k0 - B.kc);
  const double ph0 = fma(w0, y, x);
  const double f0 = ph0 - floor(ph0), fy = y - floor(y);
  const unsigned long long p0 = __double2ull_rn(f0 * 4294967296.0);
  const unsigned long long p1 = __double2ull_rn(fy * 4294967296.0);
  const double r0 = f0 - (double)p0 * 2.3283064365386963e-10;
  const double r1 = fy - (double)p1 * 2.3283064365386963e-10;
  st.acc = (uint32_t)p0 + 256u;
  st.step = (uint32_t)p1;
#pragma unroll
  for (int m = 0; m <= kRemDeg; ++m) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) s = fmaf(cf[j], B.E[j][m], s);
    st.c[m] = s;
  }
  st.c[0] += (float)(r0 - w0 * r1);
  st.c[1] += (float)r1;
#pragma unroll
  for (int m = 0; m <= kRemDeg; ++m) st.c[m] *= kTwoPiF;
  st.c[0] -= kTwoPiF;
  st.w = (float)w0;
}

__device__ __forceinline__ float mantissa_turn(uint32_t a) { return __uint_as_float((a >> 9) | 0x3f800000u); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// turns t -> 64-bit fixed point of frac(t)
__device__ __forceinline__ uint64_t frac64(double t) {
  const double x = (t - floor(t)) * 4294967296.0;  // [0, 2^32)
  const double xh = floor(x);
  const uint64_t hi = (uint64_t)xh;
  const uint64_t lo = (uint64_t)__double2ull_rn((x - xh) * 4294967296.0);  // 2^32 carries into hi
  return (hi << 32) + lo;
}

__global__ void __launch_bounds__(kTT, 1) loglike_mixed_time_kernel(LikeArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bbar[2], mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_kmax, s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, tile = tid >> 7, row = tid & 127;
  const int64_t s = (int64_t)blockIdx.x * kTT + tid;
  const bool active = s < a.n;

  // ---- per-sample set-up (FP64)
  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i)
    par[i] = (active && a.pos[i] >= 0) ? a.theta[(int64_t)a.pos[i] * a.n + s] : a.fixed[i];
  const bool valid = active && par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 &&
                     fabs(par[kChi2]) < 1.0 && par[kDl] > 0.0 && isfinite(par[kTc]) && isfinite(par[kPhic]) &&
                     isfinite(par[kRa]) && isfinite(par[kDec]) && isfinite(par[kPsi]) && isfinite(par[kIota]);
  const int nrow = a.fold ? 1 : a.n_det;
  PhaseCoeffs pc;
  int32_t kcut = 0;
  double amp = 0.0, H = 0.0;
  // Detector d enters as |P_d| c_dk e^{-i (Psi_k + 2 pi f_k dt_d - arg P_d)}: the argument of
  // the response and the delay share one 64-bit fixed-point turn counter (off, stp per bin).
  float pmag[kMaxDet];
  uint64_t off[kMaxDet], stp[kMaxDet];
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    pmag[d] = 0.f;
    off[d] = 0;
    stp[d] = 0;
  }
  if (valid) {
    const double m_sec = total_mass_seconds(par[kMc], par[kQ]);
    pc = phase_coeffs_m(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic], m_sec);
    kcut = live_bins_m(m_sec, a.f_lo, a.df, a.n_bins);
    amp = amplitude(par[kMc], par[kDl]);
    if (a.fold) {
      pmag[0] = 1.f;
      H = amp * amp * a.tfold[kcut];
    } else {
      double sp, cp, sd, cd, ss, cs;
      sincos(par[kRa] - a.gmst, &sp, &cp);
      sincos(par[kDec], &sd, &cd);
      sincos(par[kPsi], &ss, &cs);
      const double ci = cos(par[kIota]);
      for (int d = 0; d < a.n_det; ++d) {
        double fp, fc;
        antenna_trig(a.det_x[d], a.det_y[d], sp, cp, sd, cd, ss, cs, &fp, &fc);
        const double p_re = fp * 0.5 * (1.0 + ci * ci), p_im = -fc * ci;
        const double dt = delay_trig(a.det_vertex[d], sp, cp, sd, cd);
        const double p2 = p_re * p_re + p_im * p_im;
        pmag[d] = (float)sqrt(p2);
        const double arg_turns = atan2(p_im, p_re) * (1.0 / kTwoPi);
        off[d] = frac64(a.f_lo * dt - arg_turns);
        stp[d] = frac64(a.df * dt);
        H += amp * amp * p2 * a.tdet[(int64_t)d * (a.n_bins + 1) + kcut];
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < kNumBasis; ++j) pc.C[j] = 0.0;
    pc.cst = 0.0;
  }
  float cf[kNumBasis - 1];
#pragma unroll
  for (int j = 0; j < kNumBasis - 1; ++j) cf[j] = (float)pc.C[j];

  if (tid == 0) {
    s_kmax = 0;
    s_bad = 0;
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bbar[b], 1);
      tc::mbar_init(&mbar[b], 1);
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
  const int32_t nkb = (s_kmax + kKBlockBins - 1) / kKBlockBins;

  unsigned char* sA = sm + kOffA;
  unsigned char* sB = sm + kOffB;
  float4* sCd = reinterpret_cast<float4*>(sm + kOffC);
  const float* tiles = a.ttiles;
  int issued_b[2] = {0, 0}, issued_m[2] = {0, 0};  // thread 0's bookkeeping
  if (tid == 0) {
    for (int kb = 0; kb < 2 && kb < nkb; ++kb) {
      tc::mbar_expect_tx(&bbar[kb], 2 * kTileBytes);
      tc::bulk_g2s(sB + kb * 2 * kTileBytes, tiles + (int64_t)kb * 2 * 4096, kTileBytes, &bbar[kb]);
      tc::bulk_g2s(sB + kb * 2 * kTileBytes + kTileBytes, tiles + (int64_t)kb * 2 * 4096 + 4096, kTileBytes,
                   &bbar[kb]);
      ++issued_b[kb];
    }
  }

  State st;
  st.acc = 0;
  st.step = 0;
  st.w = 0.f;
#pragma unroll
  for (int m = 0; m <= kRemDeg; ++m) st.c[m] = 0.f;
  int blk = -1;
  int32_t blk_end = 0;
  bool bad = false;
  float zacc[kTimeShifts];  // this sample's Re z_j, summed over drained segments (round to nearest)
#pragma unroll
  for (int j = 0; j < kTimeShifts; ++j) zacc[j] = 0.f;
  for (int32_t kb = 0; kb < nkb; ++kb) {
    const int b = kb & 1;
    if (kb >= 2) {
      const bool ok = tc::mbar_wait(&mbar[b], (uint32_t)(((kb - 2) >> 1) & 1));
      if (__syncthreads_or(!ok || s_bad)) {
        bad = true;
        break;
      }
      if (tid == 0) {
        tc::mbar_expect_tx(&bbar[b], 2 * kTileBytes);
        tc::bulk_g2s(sB + b * 2 * kTileBytes, tiles + (int64_t)kb * 2 * 4096, kTileBytes, &bbar[b]);
        tc::bulk_g2s(sB + b * 2 * kTileBytes + kTileBytes, tiles + (int64_t)kb * 2 * 4096 + 4096, kTileBytes,
                     &bbar[b]);
        ++issued_b[b];
      }
    }
    // data tables of this K-block, per detector and bin pair: (re_k, re_k+1, im_k, im_k+1)
    float4* cst = sCd + b * kMaxDet * (kKBlockBins / 2);
    if (tid < nrow * (kKBlockBins / 2)) {
      const int d = tid / (kKBlockBins / 2), pp = tid % (kKBlockBins / 2);
      const float4 c = reinterpret_cast<const float4*>(a.cdet32)[((int64_t)d * a.n_pad16 + kb * kKBlockBins) / 2 + pp];
      cst[d * (kKBlockBins / 2) + pp] = make_float4(c.x, c.z, c.y, c.w);
    }
    __syncthreads();
    // this thread's row of the A operand: 16 bins -> 32 K values -> 8 chunks of 16 bytes.
    // Bins go in pairs (plan blocks have even starts), two lanes of f32x2 arithmetic.
    unsigned char* rowA = sA + (b * kTilesPerCta + tile) * 2 * kTileBytes + row * 128;
#pragma unroll 1
    for (int kk = 0; kk < kKBlockBins; kk += 2) {
      const int32_t k = kb * kKBlockBins + kk;
      if (k < kcut && k == blk_end) {
        ++blk;
        enter_block(a.plan, blk, pc, cf, st);
        blk_end = a.plan[blk].k1;
      }
      float2 re = f2(0.f), imc = f2(0.f), ims = f2(0.f);  // im = imc - ims
      if (k < kcut) {
        const float2 w = make_float2(st.w, st.w + 1.0f);
        float2 R = __ffma2_rn(f2(st.c[5]), w, f2(st.c[4]));
        R = __ffma2_rn(R, w, f2(st.c[3]));
        R = __ffma2_rn(R, w, f2(st.c[2]));
        R = __ffma2_rn(R, w, f2(st.c[1]));
        R = __ffma2_rn(R, w, f2(st.c[0]));
#pragma unroll
        for (int d = 0; d < kMaxDet; ++d) {
          if (d < nrow) {
            const uint32_t o0 = (uint32_t)(off[d] >> 32), o1 = (uint32_t)((off[d] + stp[d]) >> 32);
            const float2 f1 = make_float2(mantissa_turn(st.acc + o0), mantissa_turn(st.acc + st.step + o1));
            const float2 ang = __ffma2_rn(f1, f2(kTwoPiF), R);
            float2 sn, cs;
            __sincosf(ang.x, &sn.x, &cs.x);
            __sincosf(ang.y, &sn.y, &cs.y);
            const float4 c = cst[d * (kKBlockBins / 2) + (kk >> 1)];
            const float2 cx = make_float2(c.x, c.y), cy = make_float2(c.z, c.w);
            const float2 q = __fmul2_rn(f2(pmag[d]), cs), r = __fmul2_rn(f2(pmag[d]), sn);
            re = __ffma2_rn(cx, q, __ffma2_rn(cy, r, re));
            imc = __ffma2_rn(cy, q, imc);
            ims = __ffma2_rn(cx, r, ims);
          }
        }
        if (k + 1 >= kcut) {  // odd cut: the second bin of the pair is beyond the ISCO
          re.y = 0.f;
          imc.y = 0.f;
          ims.y = 0.f;
        }
      }
      st.acc += 2u * st.step;
      st.w += 2.0f;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) off[d] += 2 * stp[d];
      const float2 im = __fadd2_rn(imc, make_float2(-ims.x, -ims.y));
      float4 hi, lo;
      hi.x = tc::tf32_round(re.x); lo.x = re.x - hi.x;
      hi.y = tc::tf32_round(im.x); lo.y = im.x - hi.y;
      hi.z = tc::tf32_round(re.y); lo.z = re.y - hi.z;
      hi.w = tc::tf32_round(im.y); lo.w = im.y - hi.w;
      const int chunk = (kk >> 1) ^ (row & 7);
      *reinterpret_cast<float4*>(rowA + (chunk << 4)) = hi;
      *reinterpret_cast<float4*>(rowA + kTileBytes + (chunk << 4)) = lo;
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (!tc::mbar_wait(&bbar[b], (uint32_t)((kb >> 1) & 1))) {
        s_bad = 1;
      } else {
        tc::fence_after_sync();
        const uint32_t a_base = tc::smem_addr(sA + b * kTilesPerCta * 2 * kTileBytes);
        const uint32_t b_base = tc::smem_addr(sB + b * 2 * kTileBytes);
        const bool seg_first = (kb % kSegBlocks) == 0;
#pragma unroll
        for (int t = 0; t < kTilesPerCta; ++t)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
#pragma unroll
            for (int term = 0; term < 3; ++term) {
              // head.head into the main accumulator, the two correction terms into their own
              const uint32_t aa = a_base + t * 2 * kTileBytes + (term == 2 ? kTileBytes : 0) + ks * 32;
              const uint32_t bb = b_base + (term == 1 ? kTileBytes : 0) + ks * 32;
              const uint32_t d = tmem + t * 2 * kTimeShifts + (term == 0 ? 0 : kTimeShifts);
              const bool fresh = seg_first && ks == 0 && term <= 1;
              tc::mma_tf32(d, tc::desc_k_sw128(aa), tc::desc_k_sw128(bb), kIdesc, fresh ? 0u : 1u);
            }
        tc::commit(&mbar[b]);
        ++issued_m[b];
      }
    }
    // drain the TMEM accumulators into FP32 registers every kSegBlocks blocks (and at the end)
    if ((kb + 1) % kSegBlocks == 0 || kb == nkb - 1) {
      const bool ok = tc::mbar_wait(&mbar[b], (uint32_t)((kb >> 1) & 1));
      if (__syncthreads_or(!ok || s_bad)) {
        bad = true;
        break;
      }
      tc::fence_after_sync();
      const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(tile * 2 * kTimeShifts);
#pragma unroll
      for (int c0 = 0; c0 < kTimeShifts; c0 += 32) {
        uint32_t rm[32], rc[32];
        tc::tmem_ld32(base + c0, rm);
        tc::tmem_ld32(base + kTimeShifts + c0, rc);
#pragma unroll
        for (int i = 0; i < 32; ++i) zacc[c0 + i] += __uint_as_float(rm[i]) + __uint_as_float(rc[i]);
      }
      tc::fence_before_sync();
    }
  }
  double ll = 0.0;
  if (!bad && nkb > 0) {
    float m = -INFINITY;
#pragma unroll
    for (int j = 0; j < kTimeShifts; ++j) m = fmaxf(m, zacc[j]);
    const double g = amp * a.cscale;  // Re z_j = g * accumulator_j
    const float gf = (float)g;
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < kTimeShifts; ++j) sum += __expf(gf * (zacc[j] - m));
    ll = g * (double)m + log((double)sum / kTimeShifts) - 0.5 * H;
  } else if (!bad) {
    ll = -0.5 * H;
  }
  if (bad && tid == 0) {
    atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
    // let outstanding copies and MMAs finish (bounded) before the CTA releases its memory
    for (int b = 0; b < 2; ++b) {
      if (issued_b[b] > 0) (void)tc::mbar_wait(&bbar[b], (uint32_t)((issued_b[b] - 1) & 1), 1000000000ull);
      if (issued_m[b] > 0) (void)tc::mbar_wait(&mbar[b], (uint32_t)((issued_m[b] - 1) & 1), 1000000000ull);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<512>(tmem);
  if (active) a.out[s] = bad ? NAN : (valid ? ll : -INFINITY);
}

}  // namespace

cudaError_t launch_loglike_mixed_time(const LikeArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(loglike_mixed_time_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t blocks = (a.n + kTT - 1) / kTT;
  loglike_mixed_time_kernel<<<(unsigned)blocks, kTT, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mbis
