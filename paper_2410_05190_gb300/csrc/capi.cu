// capi.cu -- extern "C" entry points declared in include/mbis.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "marg.cuh"

using namespace mbis;

namespace {

thread_local std::string g_last_error;

mbis_status fail(mbis_ctx* ctx, mbis_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  g_last_error = msg;
  return st;
}

#define CU_TRY(ctx, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    }                                                                                            \
  } while (0)

bool is_periodic(int id) { return id == kRa || id == kPsi || id == kPhic; }

// integral of (1 + q)^(2/5) q^(-6/5) over [a, b]: composite 8-point Gauss-Legendre
double q_integral(double a, double b) {
  double x[kGL8], w[kGL8];
  gauss_legendre(kGL8, x, w);
  const int panels = 256;
  const double h = (b - a) / panels;
  double s = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double mid = a + (p + 0.5) * h;
    for (int i = 0; i < kGL8; ++i) {
      const double q = mid + 0.5 * h * x[i];
      s += 0.5 * h * w[i] * pow(1.0 + q, 0.4) * pow(q, -1.2);
    }
  }
  return s;
}

void free_tables(mbis_ctx* c) {
  dfree(c, c->d_cfold64);
  dfree(c, c->d_tfold);
  dfree(c, c->d_cdet64);
  dfree(c, c->d_tdet);
  dfree(c, c->d_cfold32);
  dfree(c, c->d_twiddle);
  dfree(c, c->d_cdet32);
  dfree(c, c->d_ttiles);
  dfree(c, c->d_plan);
  c->n_blocks = 0;
  c->tables_mode = -1;
}

DetResponse response_of(const mbis_ctx* c, int d) {
  double fp, fc;
  antenna(c->dets[d].xarm, c->dets[d].yarm, c->fixed[kRa], c->fixed[kDec], c->fixed[kPsi], c->gmst, &fp, &fc);
  const double ci = cos(c->fixed[kIota]);
  DetResponse r;
  r.pre = fp * 0.5 * (1.0 + ci * ci);
  r.pim = -fc * ci;
  r.dt = geocentre_delay(c->dets[d].vertex_m, c->fixed[kRa], c->fixed[kDec], c->gmst);
  return r;
}

bool sampled(const mbis_ctx* c, int slot) {
  for (int p = 0; p < c->P; ++p)
    if (c->ids[p] == slot) return true;
  return false;
}

// bound on |C_j| over the prior box (grid over Mc, q, chi1, chi2; 50% margin)
void coefficient_bounds(const mbis_ctx* c, double* cmax) {
  double lo[4], hi[4];
  const int slots[4] = {kMc, kQ, kChi1, kChi2};
  for (int s = 0; s < 4; ++s) {
    lo[s] = hi[s] = c->fixed[slots[s]];
    for (int p = 0; p < c->P; ++p)
      if (c->ids[p] == slots[s]) {
        lo[s] = c->lo[p];
        hi[s] = c->hi[p];
      }
  }
  for (int j = 0; j < kNumBasis; ++j) cmax[j] = 0.0;
  const int g = 5;
  for (int a = 0; a < g; ++a)
    for (int b = 0; b < g; ++b)
      for (int x = 0; x < g; ++x)
        for (int y = 0; y < g; ++y) {
          const double mc = lo[0] + (hi[0] - lo[0]) * a / (g - 1), q = lo[1] + (hi[1] - lo[1]) * b / (g - 1);
          const double c1 = lo[2] + (hi[2] - lo[2]) * x / (g - 1), c2 = lo[3] + (hi[3] - lo[3]) * y / (g - 1);
          if (!(mc > 0 && q > 0)) continue;
          const PhaseCoeffs pc = phase_coeffs(mc, q, c1, c2, 0.0, 0.0);
          for (int j = 0; j < kNumBasis; ++j) cmax[j] = std::max(cmax[j], 1.5 * std::fabs(pc.C[j]));
        }
}

mbis_status build_tables(mbis_ctx* c) {
  const bool fold = !(sampled(c, kRa) || sampled(c, kDec) || sampled(c, kPsi) || sampled(c, kIota));
  free_tables(c);
  ++c->gen;
  ++c->tables_gen;
  c->rb_use = 0;  // the relative-binning set-up belongs to the old tables
  const int32_t n = c->n_bins, nd = c->n_det;
  cudaStream_t s = c->stream;
  double* d_w = nullptr;
  if (fold) {
    DetResponse det[kMaxDet];
    for (int d = 0; d < nd; ++d) det[d] = response_of(c, d);
    CU_TRY(c, dalloc(c, &c->d_cfold64, sizeof(double2) * n));
    CU_TRY(c, dalloc(c, &c->d_tfold, sizeof(double) * (n + 1)));
    CU_TRY(c, dalloc(c, &d_w, sizeof(double) * n));
    CU_TRY(c, launch_event_tables(nd, n, c->f_lo, c->df, c->dtype, c->d_strain, c->d_psd64, 1, det, c->d_cfold64, d_w, s));
    CU_TRY(c, launch_prefix_rows(d_w, 1, n, c->d_tfold, s));
  } else {
    CU_TRY(c, dalloc(c, &c->d_cdet64, sizeof(double2) * (size_t)n * nd));
    CU_TRY(c, dalloc(c, &c->d_tdet, sizeof(double) * (size_t)(n + 1) * nd));
    CU_TRY(c, dalloc(c, &d_w, sizeof(double) * (size_t)n * nd));
    CU_TRY(c, launch_event_tables(nd, n, c->f_lo, c->df, c->dtype, c->d_strain, c->d_psd64, 0, nullptr, c->d_cdet64,
                                  d_w, s));
    CU_TRY(c, launch_prefix_rows(d_w, nd, n, c->d_tdet, s));
  }
  if (c->opts.precision == MBIS_MIXED) {
    // FP32 copies are scaled by a power of two near the largest magnitude
    const double2* src = fold ? c->d_cfold64 : c->d_cdet64;
    const int32_t rows = fold ? 1 : nd;
    double* d_max = nullptr;
    CU_TRY(c, dalloc(c, &d_max, sizeof(double)));
    CU_TRY(c, launch_max_abs(src, n * rows, d_max, s));
    double mx = 0.0;
    CU_TRY(c, cudaMemcpyAsync(&mx, d_max, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU_TRY(c, cudaStreamSynchronize(s));
    dfree(c, d_max);
    c->cscale = (mx > 0.0 && std::isfinite(mx)) ? std::ldexp(1.0, std::ilogb(mx) + 1) : 1.0;
    if (c->opts.marg & MBIS_MARG_TIME) {
      c->n_pad16 = (n + kKBlockBins - 1) / kKBlockBins * kKBlockBins;
      c->n_kb = c->n_pad16 / kKBlockBins;
      CU_TRY(c, dalloc(c, &c->d_cdet32, sizeof(float2) * (size_t)c->n_pad16 * rows));
      CU_TRY(c, launch_rows_to_f32(src, rows, n, c->n_pad16, 1.0 / c->cscale, c->d_cdet32, s));
      if (c->opts.n_tshift == kTimeShifts) {
        CU_TRY(c, dalloc(c, &c->d_ttiles, sizeof(float) * (size_t)c->n_kb * 2 * 4096));
        CU_TRY(c, launch_twiddle_tiles(n, c->f_lo, c->df, c->opts.dt_shift, c->n_kb, c->d_ttiles, s));
      }
    } else if (fold) {
      const int32_t n_pad = (n + kChunk - 1) / kChunk * kChunk;
      CU_TRY(c, dalloc(c, &c->d_cfold32, sizeof(float4) * (n_pad / 2)));
      CU_TRY(c, launch_to_f32(c->d_cfold64, n, n_pad, 1.0 / c->cscale, c->d_cfold32, s));
    }
    PlanInput pin;
    pin.f_lo = c->f_lo;
    pin.df = c->df;
    pin.n_bins = n;
    coefficient_bounds(c, pin.cmax);
    pin.tol_turns = 2e-8;
    pin.rmax_turns = 1.0;
    pin.max_block = 4096;
    pin.deg = (c->opts.marg & MBIS_MARG_TIME) ? kTimeRemDeg : kFoldRemDeg;  // the launching kernel's degree
    const std::vector<AnchorBlock> plan = plan_anchor_blocks(pin);
    c->n_blocks = (int32_t)plan.size();
    // float-float block entry when every phase term, its per-bin slope times the block
    // length, the t_c term and the constant stay below kFloatFloatMaxTurns
    double tc_max = std::fabs(c->fixed[kTc]);
    for (int p = 0; p < c->P; ++p)
      if (c->ids[p] == kTc) tc_max = std::max(std::fabs(c->lo[p]), std::fabs(c->hi[p]));
    double term_max = tc_max * (c->f_lo + c->df * n) + 1024.0;
    for (const AnchorBlock& b : plan)
      for (int j = 0; j < kNumBasis - 1; ++j)
        term_max = std::max(term_max, pin.cmax[j] * (std::fabs(b.B[j]) + std::fabs(b.dB[j]) * (b.k1 - b.k0)));
    c->ff_phase = term_max < kFloatFloatMaxTurns ? 1 : 0;
    CU_TRY(c, dalloc(c, &c->d_plan, sizeof(AnchorBlock) * plan.size()));
    CU_TRY(c, cudaMemcpyAsync(c->d_plan, plan.data(), sizeof(AnchorBlock) * plan.size(), cudaMemcpyHostToDevice, s));
    CU_TRY(c, cudaStreamSynchronize(s));  // the host plan goes out of scope
  }
  if ((c->opts.marg & MBIS_MARG_TIME) && c->opts.precision == MBIS_FP64) {
    CU_TRY(c, dalloc(c, &c->d_twiddle, sizeof(double2) * (size_t)n * c->opts.n_tshift));
    CU_TRY(c, launch_twiddles(n, c->f_lo, c->df, c->opts.n_tshift, c->opts.dt_shift, c->d_twiddle, s));
  }
  CU_TRY(c, c->pool ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
  dfree(c, d_w);
  c->tables_mode = fold ? 1 : 0;
  return MBIS_OK;
}

void summary_from_state(double m, double s1, double s2, int64_t n, mbis_summary* out) {
  out->max_logw = m;
  out->s1 = s1;
  out->s2 = s2;
  out->n = n;
  out->all_zero = !(m > -INFINITY) || !(s1 > 0.0);
  out->ess = (s2 > 0.0) ? s1 * s1 / s2 : 0.0;
  out->log_z = (m > -INFINITY && s1 > 0.0 && n > 0) ? m + log(s1) - log((double)n) : -INFINITY;
}

__global__ void central_diff_kernel(int32_t P, const double2* h, const double* steps, int64_t len, double2* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t p = blockIdx.y;
  if (i >= len || p >= P) return;
  const double2 a = h[(2 * (int64_t)p) * len + i], b = h[(2 * (int64_t)p + 1) * len + i];
  const double inv = 1.0 / (2.0 * steps[p]);
  out[(int64_t)p * len + i] = make_double2((a.x - b.x) * inv, (a.y - b.y) * inv);
}

}  // namespace

namespace mbis {
// message for mbis_last_error(NULL) from entry points defined in other files
void set_last_error(const std::string& msg) { g_last_error = msg; }

// The order in which the CTAs of a likelihood launch take its samples: longest band first
// (a permutation in scratch the context owns), for launches of kOrderMinSamples or more whose
// prior box reaches total masses with the ISCO inside the grid; *perm = null otherwise.
mbis_status sample_order(mbis_ctx* c, const LikeArgs& a, int32_t gran, cudaStream_t s, const int32_t** perm) {
  *perm = nullptr;
  if (a.n < kOrderMinSamples || !c->may_cut) return MBIS_OK;
  if (c->tperm_cap < a.n) {
    dfree(c, c->d_tperm);
    c->tperm_cap = 0;
    CU_TRY(c, dalloc(c, &c->d_tperm, sizeof(int32_t) * (size_t)a.n));
    c->tperm_cap = a.n;
  }
  if (!c->d_thist) CU_TRY(c, dalloc(c, &c->d_thist, sizeof(int32_t) * (size_t)order_keys(c->n_bins, kFoldOrderGran)));
  CU_TRY(c, launch_sample_order(a, gran, c->d_thist, c->d_tperm, s));
  *perm = c->d_tperm;
  return MBIS_OK;
}

DrawArgs make_draw_args(const mbis_ctx* c, uint64_t seed, uint64_t ctr0, int64_t n, double* theta, double* log_q,
                        double* log_prior) {
  DrawArgs a = {};
  a.P = c->P;
  double logdet = 0.0;
  for (int p = 0; p < c->P; ++p) {
    a.ids[p] = c->ids[p];
    a.mean[p] = c->mean[p];
    a.lo[p] = c->lo[p];
    a.hi[p] = c->hi[p];
    logdet += log(c->chol[p * kMaxP + p]);
  }
  std::memcpy(a.chol, c->chol, sizeof(a.chol));
  a.scale = c->scale;
  a.flags = c->prior_flags;
  a.log_mass_norm = c->log_mass_norm;
  a.log_q_const = -logdet - 0.5 * c->P * log(kTwoPi) - c->P * log(c->scale);
  a.seed = seed;
  a.ctr0 = ctr0;
  a.d_ctr0 = nullptr;
  a.n = n;
  a.theta = theta;
  a.logq = log_q;
  a.logp = log_prior;
  return a;
}

LikeArgs make_like_args(const mbis_ctx* c, int64_t n, const double* theta, double* loglike) {
  LikeArgs a = {};
  a.n = n;
  a.theta = theta;
  a.out = loglike;
  a.P = c->P;
  for (int s = 0; s < kNumSlots; ++s) a.pos[s] = -1;
  for (int p = 0; p < c->P; ++p) {
    a.ids[p] = c->ids[p];
    a.pos[c->ids[p]] = (int8_t)p;
  }
  std::memcpy(a.fixed, c->fixed, sizeof(a.fixed));
  a.marg = c->opts.marg;
  a.dmin = c->opts.dmin_mpc;
  a.dmax = c->opts.dmax_mpc;
  a.n_tshift = c->opts.n_tshift;
  a.dt_shift = c->opts.dt_shift;
  a.n_bins = c->n_bins;
  a.n_det = c->n_det;
  a.f_lo = c->f_lo;
  a.df = c->df;
  a.fold = c->tables_mode == 1;
  a.basis = c->d_basis;
  a.cfold64 = c->d_cfold64;
  a.tfold = c->d_tfold;
  a.cdet64 = c->d_cdet64;
  a.tdet = c->d_tdet;
  auto split = [](double v, float (&out)[2]) {
    out[0] = (float)v;
    out[1] = (float)(v - (double)out[0]);
  };
  for (int d = 0; d < c->n_det; ++d)
    for (int i = 0; i < 3; ++i) {
      a.det_vertex[d][i] = c->dets[d].vertex_m[i];
      a.det_x[d][i] = c->dets[d].xarm[i];
      a.det_y[d][i] = c->dets[d].yarm[i];
      split(c->dets[d].xarm[i], a.det_xf[d][i]);
      split(c->dets[d].yarm[i], a.det_yf[d][i]);
      split(-c->f_lo * c->dets[d].vertex_m[i] * kInvClight, a.det_offf[d][i]);
      split(-c->df * c->dets[d].vertex_m[i] * kInvClight, a.det_stpf[d][i]);
    }
  a.gmst = c->gmst;
  a.twiddle = c->d_twiddle;
  a.cfold32 = c->d_cfold32;
  a.cscale = c->cscale;
  a.plan = c->d_plan;
  a.n_blocks = c->n_blocks;
  a.cdet32 = c->d_cdet32;
  a.n_pad16 = c->n_pad16;
  a.ttiles = c->d_ttiles;
  a.n_kb = c->n_kb;
  a.ff_phase = c->ff_phase;
  a.err = c->d_err;
  a.gl = c->d_gl;
  a.glf = reinterpret_cast<const float*>(c->d_gl + kGLSize);
  a.dist = dist_const(c->opts.dmin_mpc, c->opts.dmax_mpc);
  return a;
}
}  // namespace mbis

mbis_status mbis::create_ctx(const mbis_event* ev, const double* psd, const mbis_detector* dets,
                             const mbis_freq_grid* grid, const mbis_options* opts, const CtxEnv& env, mbis_ctx** out) {
  if (out) *out = nullptr;
  if (!ev || !psd || !dets || !grid || !opts || !out || !ev->strain)
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: null argument");
  if (ev->n_det < 1 || ev->n_det > kMaxDet) return fail(nullptr, MBIS_E_INVALID, "mbis_create: n_det must be 1..4");
  if (ev->dtype != MBIS_C128 && ev->dtype != MBIS_C64) return fail(nullptr, MBIS_E_INVALID, "mbis_create: bad dtype");
  if (grid->n_bins < 1 || !(grid->df > 0.0) || !(grid->f_lo > 0.0))
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: grid needs n_bins >= 1, df > 0, f_lo > 0");
  if (opts->precision != MBIS_FP64 && opts->precision != MBIS_MIXED)
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: precision must be MBIS_FP64 or MBIS_MIXED");
  const uint32_t mg = opts->marg;
  if (!(mg == 0 || mg == MBIS_MARG_PHASE || mg == (MBIS_MARG_PHASE | MBIS_MARG_DISTANCE) || mg == MBIS_MARG_TIME))
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: marg must be 0, PHASE, PHASE|DISTANCE or TIME");
  if ((mg & MBIS_MARG_DISTANCE) && !(opts->dmin_mpc > 0.0 && opts->dmax_mpc > opts->dmin_mpc))
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: distance range needs 0 < dmin < dmax");
  if ((mg & MBIS_MARG_TIME) && !(opts->n_tshift >= 1 && opts->n_tshift <= 256 && opts->dt_shift > 0.0))
    return fail(nullptr, MBIS_E_INVALID, "mbis_create: time grid needs 1 <= n_tshift <= 256 and dt_shift > 0");

  mbis_ctx* c = new (std::nothrow) mbis_ctx();
  if (!c) return fail(nullptr, MBIS_E_OOM, "mbis_create: host allocation failed");
  c->n_det = ev->n_det;
  c->n_bins = grid->n_bins;
  c->dtype = ev->dtype;
  c->f_lo = grid->f_lo;
  c->df = grid->df;
  c->gmst = ev->gmst_rad;
  std::memcpy(c->fixed, ev->fixed, sizeof(c->fixed));
  std::memcpy(c->dets, dets, sizeof(mbis_detector) * ev->n_det);
  c->opts = *opts;
  c->stream = env.stream;
  c->pool = env.pool;
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->n_sms = sms > 0 ? sms : 152;
  }
  auto bail = [&](mbis_status st) {
    std::string m = c->err;
    mbis_destroy(c);
    g_last_error = m;
    return st;
  };
  cudaGetDevice(&c->device);
  const size_t nb = (size_t)c->n_bins * c->n_det;
  const size_t csz = ev->dtype == MBIS_C128 ? 16 : 8;
  cudaStream_t s = c->stream;
  cudaError_t e;
#define CREATE_TRY(call)                                                                                 \
  if ((e = (call)) != cudaSuccess) {                                                                     \
    fail(c, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA, std::string(#call) + ": " +        \
                                                                        cudaGetErrorString(e));          \
    return bail(e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA);                              \
  }
  CREATE_TRY(dalloc(c, &c->d_strain, csz * nb));
  CREATE_TRY(cudaMemcpyAsync(c->d_strain, ev->strain, csz * nb, cudaMemcpyHostToDevice, s));
  for (size_t i = 0; i < nb; ++i)
    if (!(psd[i] > 0.0) || !std::isfinite(psd[i])) {
      fail(c, MBIS_E_INVALID, "mbis_create: PSD must be positive and finite");
      return bail(MBIS_E_INVALID);
    }
  CREATE_TRY(dalloc(c, &c->d_psd64, sizeof(double) * nb));
  CREATE_TRY(cudaMemcpyAsync(c->d_psd64, psd, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
  CREATE_TRY(dalloc(c, &c->d_basis, sizeof(double) * kNumBasis * (size_t)c->n_bins));
  CREATE_TRY(launch_basis_table(c->f_lo, c->df, c->n_bins, c->d_basis, s));
  {
    // FP64 nodes / weights followed by their FP32 copy
    double gl[kGLSize];
    float glf[kGLSize];
    fill_gauss_legendre(gl);
    fill_gauss_legendre_f32(glf);
    CREATE_TRY(dalloc(c, &c->d_gl, sizeof(gl) + sizeof(glf)));
    CREATE_TRY(cudaMemcpyAsync(c->d_gl, gl, sizeof(gl), cudaMemcpyHostToDevice, s));
    CREATE_TRY(cudaMemcpyAsync(c->d_gl + kGLSize, glf, sizeof(glf), cudaMemcpyHostToDevice, s));
    CREATE_TRY(cudaStreamSynchronize(s));  // gl, glf are on this stack frame
  }
  CREATE_TRY(dalloc(c, &c->d_err, sizeof(int32_t)));
  CREATE_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));
  CREATE_TRY(dalloc(c, &c->red.partials, sizeof(double) * 2 * kReduceBlocks));
  CREATE_TRY(dalloc(c, &c->red.counter, sizeof(unsigned int)));
  CREATE_TRY(cudaMemsetAsync(c->red.counter, 0, sizeof(unsigned int), s));
  CREATE_TRY(dalloc(c, &c->red.result, sizeof(double) * 4));
  if (env.h_scratch) {
    c->h_result = env.h_scratch;
    c->own_host = false;
  } else {
    CREATE_TRY(cudaMallocHost(&c->h_result, sizeof(double) * kHostScratch));
  }
  CREATE_TRY(dalloc(c, &c->d_mom_partials, sizeof(double) * moments_partials_size(kMaxP)));
  CREATE_TRY(dalloc(c, &c->d_mom_counter, sizeof(unsigned int)));
  CREATE_TRY(cudaMemsetAsync(c->d_mom_counter, 0, sizeof(unsigned int), s));
  CREATE_TRY(dalloc(c, &c->d_mom_out, sizeof(double) * kMomentSums));
  CREATE_TRY(c->pool ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
#undef CREATE_TRY
  *out = c;
  return MBIS_OK;
}


namespace {

MomentArgs moment_args(const mbis_ctx* c) {
  MomentArgs ma = {};
  for (int p = 0; p < c->P; ++p) {
    ma.ref[p] = c->mean[p];
    ma.period[p] = c->ids[p] == kPsi ? kPi : (c->ids[p] == kRa || c->ids[p] == kPhic) ? kTwoPi : 0.0;
  }
  return ma;
}

// mean and covariance from the weighted sums [sum w, sum w d_p, sum w d_p d_q (p <= q)] of the
// offsets d from the reference point ma.ref; false when no weight is positive
bool moments_from_sums(const mbis_ctx* c, const MomentArgs& ma, const double* h, double* mean_out, double* cov_out) {
  const int32_t P = c->P;
  const double wsum = h[0];
  if (!(wsum > 0.0)) return false;
  int m = 1;
  double d[kMaxP];
  for (int p = 0; p < P; ++p) d[p] = h[m++] / wsum;
  for (int p = 0; p < P; ++p)
    for (int q = p; q < P; ++q) {
      const double v = h[m++] / wsum - d[p] * d[q];
      cov_out[p * P + q] = v;
      cov_out[q * P + p] = v;
    }
  for (int p = 0; p < P; ++p) {
    double x = ma.ref[p] + d[p];
    if (ma.period[p] > 0.0) x -= ma.period[p] * floor(x / ma.period[p]);
    mean_out[p] = x;
  }
  return true;
}

// lower Cholesky factor (row-major P x P, upper part zero); false when cov is not positive definite
bool host_cholesky(int32_t P, const double* cov, double* L) {
  for (int i = 0; i < P; ++i)
    for (int j = 0; j <= i; ++j) {
      double sum = cov[i * P + j];
      for (int k = 0; k < j; ++k) sum -= L[i * P + k] * L[j * P + k];
      if (i == j) {
        if (!(sum > 0.0)) return false;
        L[i * P + i] = sqrt(sum);
      } else {
        L[i * P + j] = sum / L[j * P + j];
      }
    }
  for (int i = 0; i < P; ++i)
    for (int j = i + 1; j < P; ++j) L[i * P + j] = 0.0;
  return true;
}

size_t round_alloc(size_t b) { return (b + 511) / 512 * 512; }

}  // namespace

size_t mbis::ctx_footprint_bytes(int32_t n_det, int32_t n_bins, int32_t dtype, const mbis_options& opts, bool fold) {
  const size_t n = (size_t)n_bins, nd = (size_t)n_det, nb = n * nd;
  size_t t = 0;
  t += round_alloc((dtype == MBIS_C128 ? 16 : 8) * nb) + round_alloc(8 * nb);  // strain, PSD
  t += round_alloc(8 * kNumBasis * n) + round_alloc(8 * kGLSize) + round_alloc(4);
  t += round_alloc(16 * kReduceBlocks) + round_alloc(4) + round_alloc(32);
  t += round_alloc(8 * (size_t)moments_partials_size(kMaxP)) + round_alloc(4) + round_alloc(8 * kMomentSums);
  const size_t rows = fold ? 1 : nd;
  t += round_alloc(16 * n * rows) + round_alloc(8 * (n + 1) * rows) + round_alloc(8 * n * rows);  // C, T, scratch
  if (opts.precision == MBIS_MIXED) {
    t += round_alloc(8);
    if (opts.marg & MBIS_MARG_TIME) {
      const size_t pad16 = (n + kKBlockBins - 1) / kKBlockBins * kKBlockBins;
      t += round_alloc(8 * pad16 * rows);
      if (opts.n_tshift == kTimeShifts) t += round_alloc(4 * (pad16 / kKBlockBins) * 2 * 4096);
    } else if (fold) {
      t += round_alloc(8 * ((n + kChunk - 1) / kChunk * kChunk));
    }
    t += round_alloc(sizeof(AnchorBlock) * (n / 2 + 2));  // the planner's blocks hold at least two bins
  }
  if ((opts.marg & MBIS_MARG_TIME) && opts.precision == MBIS_FP64) t += round_alloc(16 * n * (size_t)opts.n_tshift);
  return t;
}

mbis_status mbis::ess_begin(mbis_ctx* c, const mbis_ess_options* o, EssState* st) {
  if (!c || !o || !st) return fail(c, MBIS_E_INVALID, "ess: null argument");
  if (!c->has_metric) return fail(c, MBIS_E_STATE, "ess: call mbis_set_metric first");
  if (o->batch < 1 || o->max_samples < 1) return fail(c, MBIS_E_INVALID, "ess: batch and max_samples must be >= 1");
  mbis_reset_running(c);
  *st = EssState{};
  st->o = *o;
  st->refits_left = o->refine > 0 ? o->refine : 0;
  return MBIS_OK;
}

mbis_status mbis::ess_issue(mbis_ctx* c, EssState* st, const EssBuffers& buf, cudaStream_t s) {
  if (st->done) return fail(c, MBIS_E_STATE, "ess: the loop has finished");
  st->nb = std::min<int64_t>(st->o.batch, st->o.max_samples - st->drawn);
  st->refit = st->refits_left > 0;
  const int64_t nb = st->nb;
  const DrawArgs da = make_draw_args(c, st->o.seed, (uint64_t)(st->b * st->o.batch), nb, buf.theta, buf.log_q,
                                     buf.log_prior);
  CU_TRY(c, launch_draw(da, s));
  mbis_status r = mbis_loglike(c, nb, buf.theta, buf.loglike, s);
  if (r != MBIS_OK) return r;
  CU_TRY(c, launch_reduce(nb, buf.loglike, buf.log_prior, buf.log_q, st->refit ? buf.weights : nullptr, c->red, s));
  CU_TRY(c, cudaMemcpyAsync(c->h_result, c->red.result, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  CU_TRY(c, cudaMemcpyAsync(c->h_result + 4, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (st->refit) {
    const MomentArgs ma = moment_args(c);
    const int nm = 1 + c->P + c->P * (c->P + 1) / 2;
    CU_TRY(c, launch_moments(nb, c->P, buf.theta, buf.weights, ma, c->d_mom_partials, c->d_mom_counter,
                             c->d_mom_out, s));
    CU_TRY(c, cudaMemcpyAsync(c->h_result + 8, c->d_mom_out, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  }
  return MBIS_OK;
}

mbis_status mbis::ess_complete(mbis_ctx* c, EssState* st) {
  int32_t derr;
  std::memcpy(&derr, c->h_result + 4, sizeof(int32_t));
  if (derr != 0) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream);
    st->done = true;
    return fail(c, MBIS_E_TIMEOUT, "a device-side wait timed out in a kernel of this context");
  }
  const int64_t nb = st->nb;
  mbis_summary batch;
  summary_from_state(c->h_result[0], c->h_result[1], c->h_result[2], nb, &batch);
  st->drawn += nb;
  ++st->b;
  if (st->refit) {
    const double min_fit = 2.0 * c->P + 1.0;
    const int nm = 1 + c->P + c->P * (c->P + 1) / 2;
    const double* sums = c->h_result + 8;  // this batch's sums, weights normalised to its S1
    double pool_ess = batch.ess;
    if (st->o.refit_min_ess > min_fit) {  // pool with earlier batches of this proposal
      mbis_summary merged = batch;
      if (st->pooled > 0) mbis_merge_summaries(&st->pool, &batch, &merged);
      const double m_new = merged.max_logw;
      const double a_old = st->pooled > 0 && st->pool.max_logw > -INFINITY ? exp(st->pool.max_logw - m_new) : 0.0;
      const double a_b = batch.max_logw > -INFINITY ? batch.s1 * exp(batch.max_logw - m_new) : 0.0;
      for (int j = 0; j < nm; ++j)  // a batch or pool of zero weight adds nothing (its sums may be NaN)
        st->mom[j] = (a_old > 0.0 ? a_old * st->mom[j] : 0.0) + (a_b > 0.0 ? a_b * sums[j] : 0.0);
      st->pool = merged;
      ++st->pooled;
      pool_ess = merged.ess;
      sums = st->mom;
      if (pool_ess < st->o.refit_min_ess && st->pooled < kMaxRefitPool) {  // keep pooling
        mbis_reset_running(c);
        st->used = 0;
        st->cur = mbis_summary{};
        if (st->drawn >= st->o.max_samples) st->done = true;
        return MBIS_OK;
      }
      st->pooled = 0;
    }
    --st->refits_left;
    if (pool_ess >= min_fit) {
      const MomentArgs ma = moment_args(c);
      double mean[kMaxP], cov[kMaxP * kMaxP], L[kMaxP * kMaxP];
      if (moments_from_sums(c, ma, sums, mean, cov) && host_cholesky(c->P, cov, L)) {
        const mbis_status r =
            mbis_set_proposal(c, mean, L, st->o.refine_scale > 0.0 ? st->o.refine_scale : c->scale);
        if (r != MBIS_OK) {
          st->done = true;
          return r;
        }
      }
    }
    mbis_reset_running(c);
    st->used = 0;
    st->cur = mbis_summary{};
  } else {
    if (c->has_running) {
      mbis_summary merged;
      mbis_merge_summaries(&c->running, &batch, &merged);
      c->running = merged;
    } else {
      c->running = batch;
      c->has_running = true;
    }
    st->cur = c->running;
    st->used += nb;
    if (st->cur.ess >= st->o.ess_target) st->done = true;
  }
  if (st->drawn >= st->o.max_samples) st->done = true;
  return MBIS_OK;
}

void mbis::ess_result(const EssState& st, mbis_summary* out, int64_t* n_drawn, int64_t* n_used) {
  mbis_summary cur = st.cur;
  if (st.used == 0) summary_from_state(-INFINITY, 0.0, 0.0, 0, &cur);
  if (out) *out = cur;
  if (n_drawn) *n_drawn = st.drawn;
  if (n_used) *n_used = st.used;
}

extern "C" {

const char* mbis_version(void) { return "mbis 0.1 (sm_103a)"; }

const char* mbis_last_error(const mbis_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

mbis_status mbis_create(const mbis_event* ev, const double* psd, const mbis_detector* dets, const mbis_freq_grid* grid,
                        const mbis_options* opts, mbis_ctx** out) {
  return create_ctx(ev, psd, dets, grid, opts, CtxEnv{}, out);
}

void mbis_destroy(mbis_ctx* c) {
  if (!c) return;
  rb_free(c);
  free_tables(c);
  dfree(c, c->d_zpart);
  dfree(c, c->d_tperm);
  dfree(c, c->d_thist);
  c->tperm_cap = 0;
  dfree(c, c->d_amp);
  dfree(c, c->d_kcut);
  dfree(c, c->d_strain);
  dfree(c, c->d_psd64);
  dfree(c, c->d_basis);
  dfree(c, c->d_gl);
  dfree(c, c->d_err);
  dfree(c, c->red.partials);
  dfree(c, c->red.counter);
  dfree(c, c->red.result);
  if (c->h_result && c->own_host) cudaFreeHost(c->h_result);
  dfree(c, c->d_mom_partials);
  dfree(c, c->d_mom_counter);
  dfree(c, c->d_mom_out);
  delete c;
}

mbis_status mbis_set_metric(mbis_ctx* c, int32_t P, const int32_t* ids, const double* mean, const double* chol,
                            double scale, const double* lo, const double* hi, uint32_t flags) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_set_metric: null context");
  if (P < 1 || P > kMaxP || !ids || !mean || !chol || !lo || !hi)
    return fail(c, MBIS_E_INVALID, "mbis_set_metric: P must be 1..11 and arrays non-null");
  if (!(scale > 0.0) || !std::isfinite(scale)) return fail(c, MBIS_E_INVALID, "mbis_set_metric: scale must be > 0");
  bool seen[kNumSlots] = {};
  for (int p = 0; p < P; ++p) {
    const int id = ids[p];
    if (id < 0 || id >= kNumSlots || seen[id]) return fail(c, MBIS_E_INVALID, "mbis_set_metric: bad or repeated slot");
    seen[id] = true;
    if ((id == kPhic && (c->opts.marg & MBIS_MARG_PHASE)) || (id == kDl && (c->opts.marg & MBIS_MARG_DISTANCE)))
      return fail(c, MBIS_E_INVALID, "mbis_set_metric: a marginalised slot cannot be sampled");
    if (!(chol[p * P + p] > 0.0)) return fail(c, MBIS_E_INVALID, "mbis_set_metric: Cholesky diagonal must be > 0");
    if (!is_periodic(id) && !(lo[p] < hi[p])) return fail(c, MBIS_E_INVALID, "mbis_set_metric: need prior_lo < hi");
    if (id == kDec && (lo[p] < -kPi / 2 || hi[p] > kPi / 2))
      return fail(c, MBIS_E_INVALID, "mbis_set_metric: dec prior outside [-pi/2, pi/2]");
    if (id == kIota && (lo[p] < 0 || hi[p] > kPi))
      return fail(c, MBIS_E_INVALID, "mbis_set_metric: iota prior outside [0, pi]");
    if ((id == kMc || id == kQ || id == kDl) && !(lo[p] > 0.0))
      return fail(c, MBIS_E_INVALID, "mbis_set_metric: Mc, q and d_L priors need lo > 0");
  }
  if ((flags & MBIS_PRIOR_M1M2) && !(seen[kMc] && seen[kQ]))
    return fail(c, MBIS_E_INVALID, "mbis_set_metric: the component-mass prior needs Mc and q sampled");
  c->P = P;
  for (int p = 0; p < P; ++p) {
    c->ids[p] = ids[p];
    c->mean[p] = mean[p];
    c->lo[p] = is_periodic(ids[p]) ? 0.0 : lo[p];
    c->hi[p] = is_periodic(ids[p]) ? (ids[p] == kPsi ? kPi : kTwoPi) : hi[p];
    for (int r = 0; r < kMaxP; ++r) c->chol[p * kMaxP + r] = (r <= p && r < P) ? chol[p * P + r] : 0.0;
  }
  c->scale = scale;
  c->prior_flags = flags;
  c->log_mass_norm = 0.0;
  if (flags & MBIS_PRIOR_M1M2) {
    double mlo = 0, mhi = 0, qlo = 0, qhi = 0;
    for (int p = 0; p < P; ++p) {
      if (ids[p] == kMc) { mlo = lo[p]; mhi = hi[p]; }
      if (ids[p] == kQ) { qlo = lo[p]; qhi = hi[p]; }
    }
    c->log_mass_norm = log(0.5 * (mhi * mhi - mlo * mlo) * q_integral(qlo, qhi));
  }
  {
    // whether samples inside the prior box can end (ISCO) inside the grid: then a launch
    // orders its samples by their live bins
    double mc_hi = c->fixed[kMc], q_lo = c->fixed[kQ], q_hi = c->fixed[kQ];
    for (int p = 0; p < P; ++p) {
      if (ids[p] == kMc) mc_hi = hi[p];
      if (ids[p] == kQ) {
        q_lo = lo[p];
        q_hi = hi[p];
      }
    }
    double m_max = 0.0;
    for (const double q : {q_lo, q_hi})
      if (q > 0.0 && mc_hi > 0.0) m_max = std::max(m_max, total_mass_seconds(mc_hi, q));
    c->may_cut = m_max > 0.0 && f_isco_m(m_max) <= c->f_lo + c->df * (c->n_bins - 1);
  }
  const mbis_status st = build_tables(c);
  if (st != MBIS_OK) return st;
  c->has_metric = true;
  return MBIS_OK;
}

mbis_status mbis_draw(mbis_ctx* c, uint64_t seed, uint64_t ctr0, int64_t n, double* theta, double* log_q,
                      double* log_prior, void* stream) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_draw: null context");
  if (!c->has_metric) return fail(c, MBIS_E_STATE, "mbis_draw: call mbis_set_metric first");
  if (n < 0 || (n > 0 && !theta)) return fail(c, MBIS_E_INVALID, "mbis_draw: bad n or null theta");
  const DrawArgs a = make_draw_args(c, seed, ctr0, n, theta, log_q, log_prior);
  CU_TRY(c, launch_draw(a, static_cast<cudaStream_t>(stream)));
  return MBIS_OK;
}

mbis_status mbis_loglike(mbis_ctx* c, int64_t n, const double* theta, double* loglike, void* stream) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_loglike: null context");
  if (!c->has_metric) return fail(c, MBIS_E_STATE, "mbis_loglike: call mbis_set_metric first");
  if (n < 0 || (n > 0 && (!theta || !loglike))) return fail(c, MBIS_E_INVALID, "mbis_loglike: bad n or null buffer");
  if ((c->opts.marg & MBIS_MARG_TIME) && c->opts.precision == MBIS_MIXED && c->d_ttiles == nullptr)
    return fail(c, MBIS_E_UNSUPPORTED, "mbis_loglike: mixed-precision time marginalisation needs n_tshift = 128");
  if (c->rb_use) return mbis_rb_loglike(c, n, theta, loglike, stream);
  const LikeArgs a = make_like_args(c, n, theta, loglike);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->opts.precision == MBIS_FP64) {
    CU_TRY(c, launch_loglike_fp64(a, s));
  } else if (c->opts.marg & MBIS_MARG_TIME) {
    LikeArgs b = a;
    if (const mbis_status r = sample_order(c, a, kKBlockBins, s, &b.perm); r != MBIS_OK) return r;
    CU_TRY(c, launch_loglike_mixed_time(b, s));
  } else {
    if (!a.fold)
      return fail(c, MBIS_E_UNSUPPORTED,
                  "mbis_loglike: mixed precision with sampled sky/orientation needs MBIS_MARG_TIME");
    // a launch with fewer tiles than the device has CTA slots splits each tile's bins over
    // several CTAs (whole parts each), so small batches still fill the GPU
    LikeArgs b = a;
    const int64_t tiles = (n + kMixedThreads - 1) / kMixedThreads, slots = (int64_t)c->n_sms * 8;
    const int32_t parts = (c->n_bins + kPartBins - 1) / kPartBins;
    // the split minimises waves x (parts per piece + the set-up, ~0.1 of a part's time): a
    // 2^16-sample batch (512 tiles, 16 parts) runs 16 one-part pieces in 6.7 waves rather
    // than 2 eight-part pieces in a wave 84% full
    b.split = 1;
    if (tiles < slots && parts > 1) {
      double best = 1e300;
      for (int32_t sp = 1; sp <= parts; ++sp) {
        const double waves = std::ceil((double)(tiles * sp) / (double)slots);
        const double t = waves * (std::ceil((double)parts / sp) + 0.1);
        if (t < best) {
          best = t;
          b.split = sp;
        }
      }
    }
    if (const mbis_status r = sample_order(c, a, kFoldOrderGran, s, &b.perm); r != MBIS_OK) return r;
    if (b.split > 1) {
      if (c->split_cap < n) {
        dfree(c, c->d_zpart);
        dfree(c, c->d_amp);
        dfree(c, c->d_kcut);
        c->split_cap = 0;
        CU_TRY(c, dalloc(c, &c->d_zpart, sizeof(double2) * (size_t)parts * (size_t)n));
        CU_TRY(c, dalloc(c, &c->d_amp, sizeof(double) * (size_t)n));
        CU_TRY(c, dalloc(c, &c->d_kcut, sizeof(int32_t) * (size_t)n));
        c->split_cap = n;
      }
      b.zpart = c->d_zpart;
      b.amp_out = c->d_amp;
      b.kcut_out = c->d_kcut;
    }
    CU_TRY(c, launch_loglike_mixed(b, s));
  }
  return MBIS_OK;
}

void mbis_merge_summaries(const mbis_summary* a, const mbis_summary* b, mbis_summary* out) {
  const double m = std::max(a->max_logw, b->max_logw);
  double s1 = 0.0, s2 = 0.0;
  if (m > -INFINITY) {
    if (a->max_logw > -INFINITY) {
      const double r = exp(a->max_logw - m);
      s1 += a->s1 * r;
      s2 += a->s2 * r * r;
    }
    if (b->max_logw > -INFINITY) {
      const double r = exp(b->max_logw - m);
      s1 += b->s1 * r;
      s2 += b->s2 * r * r;
    }
  }
  summary_from_state(m, s1, s2, a->n + b->n, out);
}

mbis_status mbis_reduce(mbis_ctx* c, int64_t n, const double* loglike, const double* log_prior, const double* log_q,
                        double* weights_out, int32_t accumulate, mbis_summary* out, void* stream) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_reduce: null context");
  if (n < 0 || !out || (n > 0 && (!loglike || !log_prior || !log_q)))
    return fail(c, MBIS_E_INVALID, "mbis_reduce: bad n or null buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU_TRY(c, launch_reduce(n, loglike, log_prior, log_q, weights_out, c->red, s));
  CU_TRY(c, cudaMemcpyAsync(c->h_result, c->red.result, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  CU_TRY(c, cudaMemcpyAsync(c->h_result + 4, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CU_TRY(c, cudaStreamSynchronize(s));
  int32_t derr;
  std::memcpy(&derr, c->h_result + 4, sizeof(int32_t));
  if (derr != 0) {
    cudaMemset(c->d_err, 0, sizeof(int32_t));
    return fail(c, MBIS_E_TIMEOUT, "a device-side wait timed out in an earlier kernel of this context");
  }
  mbis_summary batch;
  summary_from_state(n > 0 ? c->h_result[0] : -INFINITY, c->h_result[1], c->h_result[2], n, &batch);
  if (n == 0) summary_from_state(-INFINITY, 0.0, 0.0, 0, &batch);
  if (accumulate) {
    if (c->has_running) {
      mbis_summary merged;
      mbis_merge_summaries(&c->running, &batch, &merged);
      c->running = merged;
    } else {
      c->running = batch;
      c->has_running = true;
    }
    *out = c->running;
  } else {
    *out = batch;
  }
  return MBIS_OK;
}

mbis_status mbis_get_running(const mbis_ctx* c, mbis_summary* out) {
  if (!c || !out) return fail(nullptr, MBIS_E_INVALID, "mbis_get_running: null argument");
  if (c->has_running)
    *out = c->running;
  else
    summary_from_state(-INFINITY, 0.0, 0.0, 0, out);
  return MBIS_OK;
}

mbis_status mbis_reset_running(mbis_ctx* c) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_reset_running: null context");
  c->has_running = false;
  c->running = mbis_summary{};
  return MBIS_OK;
}

mbis_status mbis_psd_aligo(const mbis_freq_grid* grid, double* out) {
  if (!grid || !out || grid->n_bins < 1 || !(grid->f_lo > 0.0) || !(grid->df > 0.0))
    return fail(nullptr, MBIS_E_INVALID, "mbis_psd_aligo: bad grid or null output");
  for (int32_t k = 0; k < grid->n_bins; ++k) {
    const double f = grid->f_lo + k * grid->df, x = f / 215.0, x2 = x * x;
    out[k] = 1e-49 * (pow(x, -4.14) - 5.0 / x2 + 111.0 * (1.0 - x2 + 0.5 * x2 * x2) / (1.0 + 0.5 * x2));
  }
  return MBIS_OK;
}

mbis_status mbis_inject(const mbis_freq_grid* grid, int32_t n_det, const mbis_detector* dets, const double* psd,
                        double gmst, const double* theta, uint64_t seed, int32_t add_noise, double* strain_out,
                        double* snr2_out) {
  if (!grid || !dets || !psd || !theta || !strain_out || n_det < 1 || n_det > kMaxDet || grid->n_bins < 1)
    return fail(nullptr, MBIS_E_INVALID, "mbis_inject: bad argument");
  const int32_t n = grid->n_bins;
  const size_t len = (size_t)n * n_det;
  double *d_psd = nullptr, *d_geom = nullptr, *d_par = nullptr, *d_snr = nullptr;
  double2* d_h = nullptr;
  std::vector<double> geom(9 * n_det);
  for (int d = 0; d < n_det; ++d)
    for (int i = 0; i < 3; ++i) {
      geom[9 * d + i] = dets[d].vertex_m[i];
      geom[9 * d + 3 + i] = dets[d].xarm[i];
      geom[9 * d + 6 + i] = dets[d].yarm[i];
    }
  mbis_status st = MBIS_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&d_psd, sizeof(double) * len))) break;
    if ((e = cudaMalloc(&d_geom, sizeof(double) * geom.size()))) break;
    if ((e = cudaMalloc(&d_par, sizeof(double) * kNumSlots))) break;
    if ((e = cudaMalloc(&d_snr, sizeof(double)))) break;
    if ((e = cudaMalloc(&d_h, sizeof(double2) * len))) break;
    if ((e = cudaMemcpy(d_psd, psd, sizeof(double) * len, cudaMemcpyHostToDevice))) break;
    if ((e = cudaMemcpy(d_geom, geom.data(), sizeof(double) * geom.size(), cudaMemcpyHostToDevice))) break;
    if ((e = cudaMemcpy(d_par, theta, sizeof(double) * kNumSlots, cudaMemcpyHostToDevice))) break;
    if ((e = launch_waveforms(1, d_par, n_det, n, grid->f_lo, grid->df, nullptr, d_geom, gmst, d_h, nullptr))) break;
    if ((e = launch_inner_products(1, d_h, 1, d_h, n_det, n, grid->df, d_psd, d_snr, nullptr))) break;
    if (add_noise && (e = launch_noise(n_det, n, grid->df, d_psd, seed, d_h, nullptr))) break;
    if ((e = cudaMemcpy(strain_out, d_h, sizeof(double2) * len, cudaMemcpyDeviceToHost))) break;
    double snr2 = 0.0;
    if ((e = cudaMemcpy(&snr2, d_snr, sizeof(double), cudaMemcpyDeviceToHost))) break;
    if (snr2_out) *snr2_out = snr2;
  } while (0);
  if (e != cudaSuccess)
    st = fail(nullptr, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
              std::string("mbis_inject: ") + cudaGetErrorString(e));
  cudaFree(d_psd);
  cudaFree(d_geom);
  cudaFree(d_par);
  cudaFree(d_snr);
  cudaFree(d_h);
  return st;
}

mbis_status mbis_fisher(mbis_ctx* c, const double* theta, int32_t P, const int32_t* ids, const double* steps,
                        double* gamma_out) {
  if (!c || !theta || !ids || !steps || !gamma_out || P < 1 || P > kNumSlots)
    return fail(c, MBIS_E_INVALID, "mbis_fisher: bad argument");
  for (int p = 0; p < P; ++p)
    if (ids[p] < 0 || ids[p] >= kNumSlots || !(steps[p] > 0.0))
      return fail(c, MBIS_E_INVALID, "mbis_fisher: bad slot or non-positive step");
  const int32_t n = c->n_bins, nd = c->n_det;
  const int64_t len = (int64_t)n * nd;
  std::vector<double> par(2 * P * kNumSlots), geom(9 * nd);
  for (int p = 0; p < P; ++p)
    for (int sgn = 0; sgn < 2; ++sgn) {
      double* v = &par[(2 * p + sgn) * kNumSlots];
      std::memcpy(v, theta, sizeof(double) * kNumSlots);
      v[ids[p]] += sgn == 0 ? steps[p] : -steps[p];
    }
  for (int d = 0; d < nd; ++d)
    for (int i = 0; i < 3; ++i) {
      geom[9 * d + i] = c->dets[d].vertex_m[i];
      geom[9 * d + 3 + i] = c->dets[d].xarm[i];
      geom[9 * d + 6 + i] = c->dets[d].yarm[i];
    }
  double *d_par = nullptr, *d_geom = nullptr, *d_steps = nullptr, *d_g = nullptr;
  double2 *d_h = nullptr, *d_D = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&d_par, sizeof(double) * par.size()))) break;
    if ((e = cudaMalloc(&d_geom, sizeof(double) * geom.size()))) break;
    if ((e = cudaMalloc(&d_steps, sizeof(double) * P))) break;
    if ((e = cudaMalloc(&d_g, sizeof(double) * P * P))) break;
    if ((e = cudaMalloc(&d_h, sizeof(double2) * 2 * P * len))) break;
    if ((e = cudaMalloc(&d_D, sizeof(double2) * P * len))) break;
    if ((e = cudaMemcpy(d_par, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice))) break;
    if ((e = cudaMemcpy(d_geom, geom.data(), sizeof(double) * geom.size(), cudaMemcpyHostToDevice))) break;
    if ((e = cudaMemcpy(d_steps, steps, sizeof(double) * P, cudaMemcpyHostToDevice))) break;
    if ((e = launch_waveforms(2 * P, d_par, nd, n, c->f_lo, c->df, nullptr, d_geom, c->gmst, d_h, nullptr))) break;
    dim3 grid((unsigned)((len + 255) / 256), P);
    central_diff_kernel<<<grid, 256>>>(P, d_h, d_steps, len, d_D);
    if ((e = cudaGetLastError())) break;
    if ((e = launch_inner_products(P, d_D, P, d_D, nd, n, c->df, c->d_psd64, d_g, nullptr))) break;
    if ((e = cudaMemcpy(gamma_out, d_g, sizeof(double) * P * P, cudaMemcpyDeviceToHost))) break;
  } while (0);
  cudaFree(d_par);
  cudaFree(d_geom);
  cudaFree(d_steps);
  cudaFree(d_g);
  cudaFree(d_h);
  cudaFree(d_D);
  if (e != cudaSuccess)
    return fail(c, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
                std::string("mbis_fisher: ") + cudaGetErrorString(e));
  return MBIS_OK;
}

mbis_status mbis_weighted_moments(mbis_ctx* c, int64_t n, const double* theta, const double* weights,
                                  double* mean_out, double* cov_out, void* stream) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_weighted_moments: null context");
  if (!c->has_metric) return fail(c, MBIS_E_STATE, "mbis_weighted_moments: call mbis_set_metric first");
  if (n < 0 || !mean_out || !cov_out || (n > 0 && (!theta || !weights)))
    return fail(c, MBIS_E_INVALID, "mbis_weighted_moments: bad n or null buffer");
  const int32_t P = c->P, nm = 1 + P + P * (P + 1) / 2;
  const MomentArgs ma = moment_args(c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<double> h(nm, 0.0);
  if (n > 0) {
    CU_TRY(c, launch_moments(n, P, theta, weights, ma, c->d_mom_partials, c->d_mom_counter, c->d_mom_out, s));
    CU_TRY(c, cudaMemcpyAsync(h.data(), c->d_mom_out, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
    CU_TRY(c, cudaStreamSynchronize(s));
  }
  if (!moments_from_sums(c, ma, h.data(), mean_out, cov_out))
    return fail(c, MBIS_E_INVALID, "mbis_weighted_moments: no positive weight");
  return MBIS_OK;
}

mbis_status mbis_set_proposal(mbis_ctx* c, const double* mean, const double* chol, double scale) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_set_proposal: null context");
  if (!c->has_metric) return fail(c, MBIS_E_STATE, "mbis_set_proposal: call mbis_set_metric first");
  if (!mean || !chol || !(scale > 0.0) || !std::isfinite(scale))
    return fail(c, MBIS_E_INVALID, "mbis_set_proposal: null array or scale <= 0");
  const int32_t P = c->P;
  for (int p = 0; p < P; ++p)
    if (!(chol[p * P + p] > 0.0) || !std::isfinite(mean[p]))
      return fail(c, MBIS_E_INVALID, "mbis_set_proposal: Cholesky diagonal must be > 0 and the mean finite");
  for (int p = 0; p < P; ++p) {
    c->mean[p] = mean[p];
    for (int r = 0; r < kMaxP; ++r) c->chol[p * kMaxP + r] = (r <= p && r < P) ? chol[p * P + r] : 0.0;
  }
  c->scale = scale;
  ++c->gen;
  return MBIS_OK;
}

mbis_status mbis_get_info(const mbis_ctx* c, mbis_ctx_info* out) {
  if (!c || !out) return fail(nullptr, MBIS_E_INVALID, "mbis_get_info: null argument");
  mbis_ctx_info i = {};
  i.tables = c->tables_mode;
  i.n_rows = c->tables_mode == 1 ? 1 : (c->tables_mode == 0 ? c->n_det : 0);
  i.ff_phase = c->opts.precision == MBIS_MIXED && c->tables_mode >= 0 ? c->ff_phase : -1;
  i.n_blocks = c->opts.precision == MBIS_MIXED ? c->n_blocks : 0;
  i.P = c->has_metric ? c->P : 0;
  *out = i;
  return MBIS_OK;
}

mbis_status mbis_get_proposal(const mbis_ctx* c, double* mean_out, double* chol_out, double* scale_out) {
  if (!c) return fail(nullptr, MBIS_E_INVALID, "mbis_get_proposal: null context");
  if (!c->has_metric) return fail(nullptr, MBIS_E_STATE, "mbis_get_proposal: no metric set");
  const int32_t P = c->P;
  for (int p = 0; p < P; ++p) {
    if (mean_out) mean_out[p] = c->mean[p];
    if (chol_out)
      for (int r = 0; r < P; ++r) chol_out[p * P + r] = c->chol[p * kMaxP + r];
  }
  if (scale_out) *scale_out = c->scale;
  return MBIS_OK;
}

mbis_status mbis_run_to_ess(mbis_ctx* c, const mbis_ess_options* o, double* theta, double* log_q, double* log_prior,
                            double* loglike, double* weights, mbis_summary* out, int64_t* n_drawn, int64_t* n_used,
                            void* stream) {
  if (!c || !o || !out) return fail(c, MBIS_E_INVALID, "mbis_run_to_ess: null argument");
  if (!theta || !log_q || !log_prior || !loglike || !weights)
    return fail(c, MBIS_E_INVALID, "mbis_run_to_ess: null buffer");
  EssState st;
  mbis_status r = ess_begin(c, o, &st);
  if (r != MBIS_OK) return r;
  const EssBuffers buf = {theta, log_q, log_prior, loglike, weights};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  while (!st.done) {
    if ((r = ess_issue(c, &st, buf, s)) != MBIS_OK) return r;
    CU_TRY(c, cudaStreamSynchronize(s));
    if ((r = ess_complete(c, &st)) != MBIS_OK) return r;
  }
  ess_result(st, out, n_drawn, n_used);
  return MBIS_OK;
}

}  // extern "C"
