// k_loglike_mixed.cu -- fused waveform + projection + inner-product + marginalisation
// kernel in mixed precision (Eqs. 1-3 with the marginalised forms of Sec. III).  The
// waveform h(f) is never written to memory.
//
// One thread per proposal sample, 128 samples per CTA.  The folded data table C_k (FP32,
// detectors and their fixed responses folded in) streams through shared memory in chunks
// of 512 bins by TMA bulk copies (cp.async.bulk + mbarrier, two buffers); every thread of
// the CTA reads the same bin at the same time (shared-memory broadcast).
//
// Phase per bin (anchor blocks, see plan.cpp): at the start of a block each thread forms,
// in FP64, the linear phase X + (k - kc) Y, reduces it modulo one turn and keeps it as a
// 32-bit fixed-point turn count (exact wrap-around on integer add), and forms in FP32 the
// coefficients of the degree-5 remainder polynomial.  The FP64 rounding residuals of the
// fixed-point value and slope are folded into that polynomial.  Per bin: one integer add,
// a 5-FMA Horner step, the fixed-point -> float conversion through the mantissa, one FMA
// to radians, MUFU sin/cos, and a complex FMA with C_k.  Per-chunk FP32 partial sums are
// accumulated in FP64.
#include "internal.h"
#include "marg.cuh"

namespace mbis {
namespace {

constexpr int kNbuf = 2;
constexpr float kTwoPiF = 6.28318530717958647692f;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for a phase of the barrier; give up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

struct BlockState {
  uint32_t acc, step;
  float c0, c1, c2, c3, c4, c5;
  float w;
  int32_t end;
};

__device__ __forceinline__ void enter_block(const AnchorBlock* __restrict__ plan, int blk, const PhaseCoeffs& pc,
                                            const float* cf, BlockState& st) {
  const AnchorBlock& B = plan[blk];
  double x = pc.cst, y = 0.0;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) {
    x = fma(pc.C[j], B.B[j], x);
    y = fma(pc.C[j], B.dB[j], y);
  }
  const double w0 = (double)(B.k0 - B.kc);
  const double ph0 = fma(w0, y, x);  // linear phase at the first bin of the block, turns
  const double f0 = ph0 - floor(ph0), fy = y - floor(y);
  const unsigned long long p0 = __double2ull_rn(f0 * 4294967296.0);
  const unsigned long long p1 = __double2ull_rn(fy * 4294967296.0);
  const double r0 = f0 - (double)p0 * 2.3283064365386963e-10;  // rounding residuals, turns
  const double r1 = fy - (double)p1 * 2.3283064365386963e-10;
  // +256: round rather than truncate when the top 23 bits become the float mantissa
  st.acc = (uint32_t)p0 + 256u;
  st.step = (uint32_t)p1;
  float c[kRemDeg + 1];
#pragma unroll
  for (int m = 0; m <= kRemDeg; ++m) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kNumBasis - 1; ++j) s = fmaf(cf[j], B.E[j][m], s);
    c[m] = s;
  }
  c[0] += (float)(r0 - w0 * r1);
  c[1] += (float)r1;
  // angle = 2 pi (acc / 2^32) + 2 pi R = 2 pi f1 + (2 pi R - 2 pi), f1 = 1 + acc / 2^32
  st.c0 = kTwoPiF * c[0] - kTwoPiF;
  st.c1 = kTwoPiF * c[1];
  st.c2 = kTwoPiF * c[2];
  st.c3 = kTwoPiF * c[3];
  st.c4 = kTwoPiF * c[4];
  st.c5 = kTwoPiF * c[5];
  st.w = (float)(B.k0 - B.kc);
  st.end = B.k1;
}

__global__ void __launch_bounds__(kMixedThreads, 4) loglike_mixed_fold_kernel(LikeArgs a) {
  __shared__ __align__(128) float2 sC[kNbuf][kChunk];
  __shared__ __align__(8) uint64_t bar[kNbuf];
  __shared__ int s_kmax;
  const int tid = threadIdx.x;
  const int64_t s = (int64_t)blockIdx.x * kMixedThreads + tid;
  const bool active = s < a.n;

  double par[kNumSlots];
#pragma unroll
  for (int i = 0; i < kNumSlots; ++i) par[i] = a.fixed[i];
  if (active)
    for (int p = 0; p < a.P; ++p) par[a.ids[p]] = a.theta[(int64_t)p * a.n + s];
  if (a.marg & MBIS_MARG_PHASE) par[kPhic] = 0.0;
  if (a.marg & MBIS_MARG_DISTANCE) par[kDl] = 1.0;
  const bool valid = active && par[kMc] > 0.0 && par[kQ] > 0.0 && fabs(par[kChi1]) < 1.0 &&
                     fabs(par[kChi2]) < 1.0 && par[kDl] > 0.0 && isfinite(par[kTc]) && isfinite(par[kPhic]);
  PhaseCoeffs pc;
  int32_t kcut = 0;
  double A = 0.0;
  if (valid) {
    pc = phase_coeffs(par[kMc], par[kQ], par[kChi1], par[kChi2], par[kTc], par[kPhic]);
    kcut = live_bins(par[kMc], par[kQ], a.f_lo, a.df, a.n_bins);
    A = amplitude(par[kMc], par[kDl]);
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
    for (int b = 0; b < kNbuf; ++b) mbar_init(&bar[b], 1);
    mbar_fence_init();
  }
  __syncthreads();
  atomicMax(&s_kmax, kcut);
  __syncthreads();
  const int32_t kmax = s_kmax;
  const int32_t nch = (kmax + kChunk - 1) / kChunk;
  constexpr uint32_t kBytes = kChunk * sizeof(float2);
  int issued[kNbuf] = {};  // copies issued per buffer (thread 0)
  if (tid == 0) {
    for (int b = 0; b < kNbuf && b < nch; ++b) {
      mbar_expect_tx(&bar[b], kBytes);
      bulk_copy_g2s(sC[b], a.cfold32 + (int64_t)b * kChunk, kBytes, &bar[b]);
      ++issued[b];
    }
  }

  double Zr = 0.0, Zi = 0.0;
  BlockState st;
  st.end = 0;
  int blk = -1;
  bool timed_out = false;
  for (int32_t ch = 0; ch < nch; ++ch) {
    const int b = ch % kNbuf;
    const bool got = mbar_wait_bounded(&bar[b], (uint32_t)((ch / kNbuf) & 1));
    if (__syncthreads_or(!got)) {
      timed_out = true;
      break;
    }
    const float2* __restrict__ cb = sC[b];
    const int32_t kb = ch * kChunk, ke = min(kb + kChunk, kmax);
    float zr = 0.f, zi = 0.f;
    int32_t k = kb;
    while (k < ke) {
      if (k == st.end) {
        ++blk;
        if (k < kcut) enter_block(a.plan, blk, pc, cf, st);
        st.end = a.plan[blk].k1;
      }
      const int32_t seg_end = min(ke, st.end);
      const int32_t my_end = min(seg_end, kcut);
      uint32_t acc = st.acc;
      float w = st.w;
      const uint32_t step = st.step;
      const float c0 = st.c0, c1 = st.c1, c2 = st.c2, c3 = st.c3, c4 = st.c4, c5 = st.c5;
#pragma unroll 4
      for (int32_t kk = k; kk < my_end; ++kk) {
        const float R = fmaf(fmaf(fmaf(fmaf(fmaf(c5, w, c4), w, c3), w, c2), w, c1), w, c0);
        const float f1 = __uint_as_float((acc >> 9) | 0x3f800000u);
        const float ang = fmaf(f1, kTwoPiF, R);
        float sn, cs;
        __sincosf(ang, &sn, &cs);
        const float2 c = cb[kk - kb];
        zr = fmaf(c.x, cs, fmaf(c.y, sn, zr));
        zi = fmaf(c.y, cs, fmaf(-c.x, sn, zi));
        acc += step;
        w += 1.0f;
      }
      // the state now stands at my_end; threads past their cut never use it again
      st.acc = acc;
      st.w = w;
      k = seg_end;
    }
    Zr += (double)zr;
    Zi += (double)zi;
    __syncthreads();  // every thread is done with buffer b
    if (tid == 0 && ch + kNbuf < nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[b], kBytes);
      bulk_copy_g2s(sC[b], a.cfold32 + (int64_t)(ch + kNbuf) * kChunk, kBytes, &bar[b]);
      ++issued[b];
    }
  }
  if (timed_out) {
    if (tid == 0) {
      atomicExch(a.err, (int32_t)MBIS_E_TIMEOUT);
      // let the last copy issued into each buffer land (bounded) before the CTA's shared
      // memory is released
      for (int bb = 0; bb < kNbuf; ++bb)
        if (issued[bb] > 0) (void)mbar_wait_bounded(&bar[bb], (uint32_t)((issued[bb] - 1) & 1));
    }
    if (active) a.out[s] = NAN;
    return;
  }
  if (!active) return;
  if (!valid) {
    a.out[s] = -INFINITY;
    return;
  }
  const double zr = A * a.cscale * Zr, zi = A * a.cscale * Zi;
  const double H = A * A * a.tfold[kcut];
  double ll;
  if (a.marg == 0) {
    ll = zr - 0.5 * H;
  } else if (a.marg == MBIS_MARG_PHASE) {
    ll = log_i0(hypot(zr, zi)) - 0.5 * H;
  } else {
    ll = log_distance_marginal(hypot(zr, zi), H, a.dmin, a.dmax, a.gl);
  }
  a.out[s] = ll;
}

}  // namespace

cudaError_t launch_loglike_mixed(const LikeArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t blocks = (a.n + kMixedThreads - 1) / kMixedThreads;
  loglike_mixed_fold_kernel<<<(unsigned)blocks, kMixedThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mbis
