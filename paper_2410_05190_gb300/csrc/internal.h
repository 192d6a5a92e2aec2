// internal.h -- context layout and kernel launchers of the CUDA path (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mbis.h"
#include "marg.cuh"
#include "physics.cuh"

namespace mbis {

constexpr int kMaxDet = 4;
constexpr int kMaxP = 11;
constexpr int kRemDegMax = 5;       // largest degree of the FP32 remainder polynomial per anchor block
// The degree each kernel family runs at (the plan of a context is built for its kernel's):
// a lower degree saves per-bin FMAs at the cost of shorter blocks, which pays in the folded
// kernel (one block entry per block) but not in the time-marginalised one (whose block entry
// also re-anchors every detector's turn counter).
constexpr int kFoldRemDeg = 4;
constexpr int kTimeRemDeg = 5;
constexpr int kChunk = 512;         // bins per shared-memory chunk of the mixed kernel
// The folded kernel sums the overlap in fixed parts of the grid, kPartChunks chunks each,
// one float pair per part added in order: the sum does not depend on how many CTAs share a
// tile's bins (small launches split them to fill the GPU).
constexpr int kPartChunks = 16;
constexpr int kPartBins = kPartChunks * kChunk;
constexpr int kMixedThreads = 128;  // samples per CTA of the mixed kernel
constexpr int kBatchCtasPerSm = 7;  // resident CTAs per SM of the persistent multi-event launch
constexpr int kReduceBlocks = 608;  // 4 x 152 SMs
constexpr int kReduceThreads = 256;

// Anchor block of the mixed-precision phase: bins [k0, k1) expanded about bin kc.
//   Psi(f_k)/2pi = [cst + sum_j C_j B_j(f_c)] + (k - kc) [sum_j C_j dB_j] + sum_j C_j R_j(k - kc)
// with R_j(w) ~ sum_m E[j][m] w^m the remainder of basis j beyond its tangent at f_c.
struct AnchorBlock {
  int32_t k0, k1, kc, pad;
  double B[kNumBasis];     // basis_j(f_kc)
  double dB[kNumBasis];    // basis_j'(f_kc) * df
  float E[kNumBasis - 1][kRemDegMax + 1];  // basis 8 (f) is linear: no remainder; degree of the plan
  // B and dB as unevaluated float pairs for the float-float block entry, one 16-byte vector
  // per basis function: (hi of B_j, lo of B_j, hi of dB_j, lo of dB_j)
  float4 Bq[kNumBasis];
};
static_assert(offsetof(AnchorBlock, E) % 16 == 0 && offsetof(AnchorBlock, Bq) % 16 == 0 &&
                  sizeof(AnchorBlock) % 16 == 0,
              "anchor-block vectors are 16-byte aligned");

// Events whose phase terms stay below this many turns may enter anchor blocks in float-float
// arithmetic (~2^-44 relative) instead of FP64.
constexpr double kFloatFloatMaxTurns = 65536.0;

struct DetResponse {
  double pre, pim;  // P_det = F+ (1 + cos^2 i)/2 - i Fx cos i
  double dt;        // geocentre delay, s
};

// Arguments shared by the likelihood kernels.
struct LikeArgs {
  int64_t n;
  const double* theta;  // [P][n]
  double* out;          // [n]
  int32_t P;
  int32_t ids[kMaxP];
  int8_t pos[kNumSlots];      // row of slot s in theta, or -1 when the slot is fixed
  double fixed[kNumSlots];
  uint32_t marg;
  double dmin, dmax;
  int32_t n_tshift;
  double dt_shift;
  int32_t n_bins, n_det;
  double f_lo, df;
  int32_t fold;               // extrinsics fixed: detectors folded into one table
  // FP64 tables
  const double* basis;        // [9][n_bins]
  const double2* cfold64;     // [n_bins] (fold)
  const double* tfold;        // [n_bins + 1] (fold) prefix sums for <h|h>
  const double2* cdet64;      // [n_det][n_bins] (non-fold)
  const double* tdet;         // [n_det][n_bins + 1]
  double det_vertex[kMaxDet][3], det_x[kMaxDet][3], det_y[kMaxDet][3];
  // the same as float pairs (hi, lo) for the float-float sky set-up of the time kernel: the
  // arms, and -f_lo r / c and -df r / c (turns at the first bin and per bin, per unit of
  // the source direction)
  float det_xf[kMaxDet][3][2], det_yf[kMaxDet][3][2], det_offf[kMaxDet][3][2], det_stpf[kMaxDet][3][2];
  double gmst;
  const double2* twiddle;     // TIME: [n_bins][n_tshift] (cos, sin) of 2 pi f_k tau_j
  // mixed tables
  const float4* cfold32;      // [n_pad / 2] bin pairs (re_k, re_k+1, im_k, im_k+1), scaled by 1 / cscale
  double cscale;
  const AnchorBlock* plan;
  int32_t n_blocks;
  const float2* cdet32;       // TIME, mixed: [n_rows][n_pad16] per-detector (or folded) tables / cscale,
                              // bin pairs interleaved (re_k, re_k+1, im_k, im_k+1)
  int32_t n_pad16;            // row length of cdet32 (multiple of 16)
  const float* ttiles;        // TIME, mixed: [n_kb][2][4096] swizzled twiddle head / tail tiles
  int32_t n_kb;               // K-blocks of 16 bins covering n_bins
  int32_t ff_phase;           // block entry in float-float (phase terms below kFloatFloatMaxTurns)
  int32_t* err;               // device error word (timeouts)
  const double* gl;           // Gauss-Legendre nodes / weights (marg.cuh layout)
  const float* glf;           // the same nodes / weights in FP32 (mixed-precision marginal)
  DistConst dist;             // distance-marginal constants of [dmin, dmax]
  // folded kernel split over CTAs (split > 1): per-part overlap sums and the per-sample
  // amplitude (negative: outside the model) and ISCO cut, read by the epilogue kernel
  int32_t split;
  double2* zpart;             // [n_parts][n]
  double* amp_out;            // [n]
  int32_t* kcut_out;          // [n]
  // mixed: the order in which CTAs take the samples (slot i evaluates sample perm[i]), most
  // live bins first; null: sample i in slot i
  const int32_t* perm;
};

struct DrawArgs {
  int32_t P;
  int32_t ids[kMaxP];
  double mean[kMaxP];
  double chol[kMaxP * kMaxP];
  double scale;
  double lo[kMaxP], hi[kMaxP];
  uint32_t flags;
  double log_mass_norm;  // ln of the (Mc, q) volume of the flat-in-(m1, m2) prior
  double log_q_const;    // -sum ln L_pp - (P/2) ln 2pi - P ln s
  uint64_t seed, ctr0;
  const uint64_t* d_ctr0;  // when set, the counter base is read from device memory (graph replays)
  int64_t n;
  double* theta;
  double* logq;
  double* logp;
};

// one work item of the persistent multi-event likelihood launch
struct BatchItem {
  int32_t ev, tile;
};

// kernel launchers (each returns cudaGetLastError() of its launch)
cudaError_t launch_basis_table(double f_lo, double df, int32_t n, double* out, cudaStream_t s);
// Samples per launch from which the mixed likelihood kernels take the samples in order of
// their live bins (longest band first); gran: the bins of one key (16 for the K-blocks of
// the time-marginalised kernel, a bin pair for the folded kernel).  hist (order_keys ints)
// and perm (n ints) are scratch of the caller; slot i of the launch evaluates perm[i].
constexpr int64_t kOrderMinSamples = 4096;
constexpr int32_t kFoldOrderGran = 2;
int32_t order_keys(int32_t n_bins, int32_t gran);
cudaError_t launch_sample_order(const LikeArgs& a, int32_t gran, int32_t* hist, int32_t* perm, cudaStream_t s);
cudaError_t launch_twiddles(int32_t n, double f_lo, double df, int32_t J, double dt, double2* out, cudaStream_t s);
cudaError_t launch_rows_to_f32(const double2* c, int32_t rows, int32_t n, int32_t n_pad, double inv_scale,
                               float2* out, cudaStream_t s);
cudaError_t launch_twiddle_tiles(int32_t n, double f_lo, double df, double dt, int32_t n_kb, float* out,
                                 cudaStream_t s);
cudaError_t launch_loglike_mixed_time(const LikeArgs& a, cudaStream_t s);

struct MomentArgs {
  double ref[kMaxP];     // offsets are taken from this point
  double period[kMaxP];  // > 0 for periodic slots (offsets wrapped into [-period/2, period/2))
};
int moments_partials_size(int32_t P);
cudaError_t launch_moments(int64_t n, int32_t P, const double* theta, const double* w, const MomentArgs& ma,
                           double* partials, unsigned int* counter, double* out, cudaStream_t s);

constexpr int kTimeShifts = 128;  // shifts of the tensor-core time marginalisation (MMA N)
constexpr int kKBlockBins = 16;   // bins per K-block of the time-shift contraction
cudaError_t launch_event_tables(int32_t n_det, int32_t n_bins, double f_lo, double df, int32_t dtype,
                                const void* strain, const double* psd, int32_t fold, const DetResponse* det,
                                double2* c_out, double* w_out, cudaStream_t s);
cudaError_t launch_prefix_rows(const double* w, int32_t rows, int32_t n, double* T, cudaStream_t s);
cudaError_t launch_max_abs(const double2* c, int32_t n, double* out, cudaStream_t s);
cudaError_t launch_to_f32(const double2* c, int32_t n, int32_t n_pad, double inv_scale, float4* out, cudaStream_t s);
cudaError_t launch_draw(const DrawArgs& a, cudaStream_t s);
cudaError_t launch_loglike_fp64(const LikeArgs& a, cudaStream_t s);
cudaError_t launch_loglike_mixed(const LikeArgs& a, cudaStream_t s);
// items of events that all enter anchor blocks in float-float (ff) or all in FP64
// tile: samples per CTA (64, 128 or 256); the grid's CTAs per SM at most batch_ctas_per_sm(tile)
cudaError_t launch_loglike_mixed_batch(const LikeArgs* args, const BatchItem* items, int32_t n_items, int32_t* next,
                                      int32_t grid, bool ff, int32_t tile, cudaStream_t s);
int32_t batch_ctas_per_sm(int32_t tile);

// two-pass weight reduction; partials / counter / result are device scratch
struct ReduceScratch {
  double* partials;       // [2 * kReduceBlocks]
  unsigned int* counter;  // [1], zero between calls
  double* result;         // [4]: m, s1, s2, n
};
cudaError_t launch_reduce(int64_t n, const double* loglike, const double* logp, const double* logq,
                          double* weights, const ReduceScratch& scr, cudaStream_t s);

// waveform helpers (FP64): strain of n_par parameter vectors, and inner products
cudaError_t launch_waveforms(int32_t n_par, const double* par /*[n_par][11] device*/, int32_t n_det, int32_t n_bins,
                             double f_lo, double df, const DetResponse* unused, const double* det_geom /*device*/,
                             double gmst, double2* h_out /*[n_par][n_det][n_bins]*/, cudaStream_t s);
cudaError_t launch_noise(int32_t n_det, int32_t n_bins, double df, const double* psd, uint64_t seed, double2* h_io,
                         cudaStream_t s);
cudaError_t launch_inner_products(int32_t n_a, const double2* a, int32_t n_b, const double2* b, int32_t n_det,
                                  int32_t n_bins, double df, const double* psd, double* out /*[n_a][n_b]*/,
                                  cudaStream_t s);

// host-side anchor planning of the mixed kernel
struct PlanInput {
  double f_lo, df;
  int32_t n_bins;
  double cmax[kNumBasis];  // bound on |C_j| over the prior
  double tol_turns;        // bound on the fit error of the phase
  double rmax_turns;       // bound on |remainder| kept in FP32
  int32_t max_block;
  int32_t deg;             // degree of the remainder polynomials (<= kRemDegMax)
};
std::vector<AnchorBlock> plan_anchor_blocks(const PlanInput& in);

void set_last_error(const std::string& msg);



}  // namespace mbis

struct mbis_ctx;
namespace mbis {
constexpr int kHostScratch = 8 + 1 + kMaxP + kMaxP * (kMaxP + 1) / 2;
constexpr int kMomentSums = 1 + kMaxP + kMaxP * (kMaxP + 1) / 2;

// where a context's memory comes from (defaults: plain cudaMalloc, legacy stream, own pinned scratch)
struct CtxEnv {
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  double* h_scratch = nullptr;  // caller-owned pinned host memory of kHostScratch doubles, or null
};
mbis_status create_ctx(const mbis_event* ev, const double* psd, const mbis_detector* dets,
                       const mbis_freq_grid* grid, const mbis_options* opts, const CtxEnv& env, mbis_ctx** out);
// upper bound on the device bytes of a context (tables for a proposal over the given slots)
size_t ctx_footprint_bytes(int32_t n_det, int32_t n_bins, int32_t dtype, const mbis_options& opts, bool fold);

// The ESS-target loop as a state machine: issue() enqueues one batch (draws, likelihoods,
// weights, and for refit batches the weighted moments) on a stream without waiting;
// complete() reads its results once the stream has finished it.
struct EssBuffers {
  double *theta, *log_q, *log_prior, *loglike, *weights;
};
struct EssState {
  mbis_ess_options o = {};
  int64_t b = 0, drawn = 0, used = 0, nb = 0;
  int refits_left = 0;
  bool refit = false;  // the batch in flight adapts the proposal
  bool done = false;
  mbis_summary cur = {};
  // refit pool: moment sums of the refit batches drawn from the current proposal, each
  // scaled to the pool's weight scale exp(pool.max_logw)
  int pooled = 0;
  mbis_summary pool = {};
  double mom[1 + kMaxP + kMaxP * (kMaxP + 1) / 2] = {};
};
constexpr int kMaxRefitPool = 16;  // batches pooled for one refit at most
mbis_status ess_begin(mbis_ctx* c, const mbis_ess_options* o, EssState* st);
mbis_status ess_issue(mbis_ctx* c, EssState* st, const EssBuffers& buf, cudaStream_t s);
mbis_status ess_complete(mbis_ctx* c, EssState* st);
void ess_result(const EssState& st, mbis_summary* out, int64_t* n_drawn, int64_t* n_used);

DrawArgs make_draw_args(const mbis_ctx* c, uint64_t seed, uint64_t ctr0, int64_t n, double* theta, double* log_q,
                        double* log_prior);
LikeArgs make_like_args(const mbis_ctx* c, int64_t n, const double* theta, double* loglike);
mbis_status sample_order(mbis_ctx* c, const LikeArgs& a, int32_t gran, cudaStream_t s, const int32_t** perm);
void rb_free(mbis_ctx* c);
}  // namespace mbis

// the context behind the opaque handle
struct mbis_ctx {
  int32_t n_det = 0, n_bins = 0, dtype = 0;
  double f_lo = 0, df = 0, gmst = 0;
  double fixed[mbis::kNumSlots] = {};
  mbis_detector dets[mbis::kMaxDet] = {};
  mbis_options opts = {};
  int device = 0;
  // allocation environment: with a pool, device memory is stream-ordered on `stream` and
  // nothing in the context's life synchronises the whole device
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  bool own_host = true;   // h_result allocated (pinned) by the context
  size_t dev_bytes = 0;   // device bytes the context holds
  size_t dev_peak = 0;    // high-water mark of dev_bytes
  std::vector<std::pair<void*, size_t>> allocs;
  void* d_strain = nullptr;
  double* d_psd64 = nullptr;  // [n_det][n_bins]
  // proposal
  bool has_metric = false;
  int32_t P = 0;
  int32_t ids[mbis::kMaxP] = {};
  double mean[mbis::kMaxP] = {}, chol[mbis::kMaxP * mbis::kMaxP] = {}, lo[mbis::kMaxP] = {}, hi[mbis::kMaxP] = {};
  double scale = 1.0;
  uint32_t prior_flags = 0;
  double log_mass_norm = 0.0;
  // tables
  int32_t tables_mode = -1;  // -1 none, 1 fold, 0 per-detector
  uint64_t gen = 0;          // bumped whenever the tables or the proposal change (batches re-capture)
  uint64_t tables_gen = 0;   // bumped whenever the tables are rebuilt (mbis_set_metric)
  int32_t n_sms = 0;         // SMs of the context's device
  // scratch of split folded launches (grown on demand)
  double2* d_zpart = nullptr;
  double* d_amp = nullptr;
  int32_t* d_kcut = nullptr;
  int64_t split_cap = 0;     // samples x parts the scratch holds
  // scratch of a launch's sample order (grown on demand)
  int32_t* d_tperm = nullptr;
  int32_t* d_thist = nullptr;
  int64_t tperm_cap = 0;
  bool may_cut = false;      // the prior box reaches total masses whose ISCO lies inside the grid
  double* d_basis = nullptr;
  double2* d_cfold64 = nullptr;
  double* d_tfold = nullptr;
  double2* d_cdet64 = nullptr;
  double* d_tdet = nullptr;
  float4* d_cfold32 = nullptr;
  double2* d_twiddle = nullptr;  // TIME marginalisation, FP64
  float2* d_cdet32 = nullptr;    // TIME marginalisation, mixed: FP32 tables
  float* d_ttiles = nullptr;     // TIME marginalisation, mixed: twiddle tiles
  int32_t n_pad16 = 0, n_kb = 0;
  int32_t ff_phase = 0;
  double cscale = 1.0;
  mbis::AnchorBlock* d_plan = nullptr;
  int32_t n_blocks = 0;
  int32_t* d_err = nullptr;
  double* d_gl = nullptr;
  // relative binning about a fiducial (mbis_rb_setup)
  int32_t rb_n = 0;                 // coarse bins (0: not set up)
  uint64_t rb_gen = 0;              // tables generation the summary data belong to
  int32_t rb_use = 0;               // mbis_loglike evaluates the relative-binning likelihood
  int32_t* d_rb_edges = nullptr;    // [rb_n + 1] bin indices of the edges
  void* d_rb_rec = nullptr;         // [rb_n + 1] 48-byte edge records (k_rb.cu)
  void* d_rb_q = nullptr;           // [rb_n] float2 q_b / scale (k_rb.cu)
  double* d_rb_prefix = nullptr;    // [4][n_bins + 1] prefix sums of W, (f - f_lo) W (re, im)
  double rb_scale = 1.0;
  double rb_C0[mbis::kNumBasis] = {}, rb_cst0 = 0.0;
  // reduction scratch
  mbis::ReduceScratch red = {};
  double* h_result = nullptr;  // pinned host scratch, kHostScratch doubles: [0..3] reduction, [4] error word,
                               // [8..] weighted-moment sums
  // weighted-moment scratch (proposal refits)
  double* d_mom_partials = nullptr;
  unsigned int* d_mom_counter = nullptr;
  double* d_mom_out = nullptr;
  mbis_summary running = {};
  bool has_running = false;
  std::string err;
};

namespace mbis {

// Device memory of a context: stream-ordered from the context's pool when it has one
// (no device-wide synchronisation), plain cudaMalloc / cudaFree otherwise.
template <typename T>
cudaError_t dalloc(mbis_ctx* c, T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&q, bytes, c->pool, c->stream) : cudaMalloc(&q, bytes);
  if (e == cudaSuccess) {
    *p = static_cast<T*>(q);
    c->dev_bytes += bytes;
    c->dev_peak = std::max(c->dev_peak, c->dev_bytes);
    c->allocs.push_back({q, bytes});
  }
  return e;
}

template <typename T>
void dfree(mbis_ctx* c, T*& p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i].first == (void*)p) {
      c->dev_bytes -= c->allocs[i].second;
      c->allocs.erase(c->allocs.begin() + i);
      break;
    }
  if (c->pool)
    cudaFreeAsync((void*)p, c->stream);
  else
    cudaFree((void*)p);
  p = nullptr;
}

}  // namespace mbis
