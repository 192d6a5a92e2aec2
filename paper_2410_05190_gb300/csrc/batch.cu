// batch.cu -- many events in one persistent likelihood launch, one CUDA graph per step.
//
// Events of uneven size (frequency grids of 2k-128k bins, 2 or 3 detectors, 2^14-2^20
// samples) share the GPU in one persistent launch per block-entry arithmetic (float-float
// or FP64; most events take the first): their 128-sample tiles form a work list, ordered
// longest first (estimated live bins), that a persistent grid of CTAs consumes through a
// device counter.  One step -- upload of the Philox counters, the draws of every
// event, the persistent likelihood launch, the two-pass reduction of every event and the
// copy of the summaries to pinned host memory -- is captured once in a CUDA graph and
// replayed.  The tile shape (samples per CTA) and the size of the persistent grid are picked
// by timing candidates (autotuner).
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace mbis;

struct mbis_batch {
  int32_t n = 0;
  std::vector<mbis_ctx*> ctx;
  std::vector<uint64_t> gen;  // each context's generation when the launch arguments were made
  std::vector<int64_t> ns;
  std::vector<uint64_t> seeds;
  std::vector<double*> theta, logq, logp, ll;
  // per event: the order in which the tiles take its samples (longest band first; null when
  // its prior box cannot end inside the grid or it has few samples) and its key counts
  std::vector<int32_t*> perm, hist;
  std::vector<LikeArgs> hargs;  // host copies of the launch arguments
  LikeArgs* d_args = nullptr;
  BatchItem* d_items = nullptr;  // float-float-entry events' tiles first, then FP64-entry ones
  int32_t n_items = 0, n_ff = 0;
  int32_t tile = kMixedThreads;  // samples per CTA of the persistent launch (64, 128 or 256)
  int64_t items_cap = 0;         // work items d_items holds (the count at the smallest tile)
  int32_t* d_next = nullptr;     // one work counter per group
  uint64_t* d_ctr = nullptr;
  uint64_t* h_ctr = nullptr;  // pinned
  double* h_res = nullptr;    // pinned, 4 per event
  int32_t grid = 152 * kBatchCtasPerSm;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace {

mbis_status berr(mbis_status st, const std::string& m) {
  set_last_error(m);
  return st;
}

#define B_TRY(call)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return berr(e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,                   \
                  std::string("mbis_batch: ") + #call + ": " + cudaGetErrorString(e_));        \
  } while (0)

// The work list: every event's 128-sample tiles, longest first (live bins at the proposal
// mean), in two groups by block-entry arithmetic -- each group runs in its own persistent
// launch.  Within an event whose prior box reaches cuts inside the grid the tiles take the
// samples longest band first (a permutation made after the draws of each step).  Rebuilt
// when a context is re-targeted.
mbis_status build_items(mbis_batch* b) {
  struct Cost {
    double cost;
    BatchItem item;
  };
  std::vector<Cost> g[2];
  for (int i = 0; i < b->n; ++i) {
    const mbis_ctx* c = b->ctx[i];
    double mc = c->fixed[kMc], q = c->fixed[kQ];
    for (int p = 0; p < c->P; ++p) {
      if (c->ids[p] == kMc) mc = c->mean[p];
      if (c->ids[p] == kQ) q = c->mean[p];
    }
    const double live = (double)live_bins(mc, q > 0 ? q : 1.0, c->f_lo, c->df, c->n_bins);
    const int32_t tiles = (int32_t)((b->ns[i] + b->tile - 1) / b->tile);
    for (int32_t t = 0; t < tiles; ++t) g[c->ff_phase ? 0 : 1].push_back({live, {i, t}});
  }
  std::vector<BatchItem> list;
  for (auto& v : g) {
    std::stable_sort(v.begin(), v.end(), [](const Cost& x, const Cost& y) { return x.cost > y.cost; });
    for (const Cost& c : v) list.push_back(c.item);
  }
  b->n_ff = (int32_t)g[0].size();
  if ((int64_t)list.size() > b->items_cap) return berr(MBIS_E_STATE, "mbis_batch: work list too long");
  b->n_items = (int32_t)list.size();
  B_TRY(cudaMemcpy(b->d_items, list.data(), sizeof(BatchItem) * list.size(), cudaMemcpyHostToDevice));
  return MBIS_OK;
}

cudaError_t launch_items(mbis_batch* b, cudaStream_t s) {
  cudaError_t e = launch_loglike_mixed_batch(b->d_args, b->d_items, b->n_ff, b->d_next, b->grid, true, b->tile, s);
  if (e == cudaSuccess)
    e = launch_loglike_mixed_batch(b->d_args, b->d_items + b->n_ff, b->n_items - b->n_ff, b->d_next + 1, b->grid,
                                   false, b->tile, s);
  return e;
}

// launch arguments of event i, with its sample order when it has one
LikeArgs batch_args(const mbis_batch* b, int i) {
  LikeArgs a = make_like_args(b->ctx[i], b->ns[i], b->theta[i], b->ll[i]);
  a.perm = b->perm[i];
  return a;
}

// enqueue one step on b->stream (also used inside stream capture)
mbis_status enqueue_step(mbis_batch* b) {
  B_TRY(cudaMemcpyAsync(b->d_ctr, b->h_ctr, sizeof(uint64_t) * b->n, cudaMemcpyHostToDevice, b->stream));
  for (int i = 0; i < b->n; ++i) {
    DrawArgs da = make_draw_args(b->ctx[i], b->seeds[i], 0, b->ns[i], b->theta[i], b->logq[i], b->logp[i]);
    da.d_ctr0 = b->d_ctr + i;
    B_TRY(launch_draw(da, b->stream));
    if (b->perm[i]) B_TRY(launch_sample_order(b->hargs[i], kFoldOrderGran, b->hist[i], b->perm[i], b->stream));
  }
  B_TRY(launch_items(b, b->stream));
  for (int i = 0; i < b->n; ++i) {
    B_TRY(launch_reduce(b->ns[i], b->ll[i], b->logp[i], b->logq[i], nullptr, b->ctx[i]->red, b->stream));
    B_TRY(cudaMemcpyAsync(b->h_res + 4 * i, b->ctx[i]->red.result, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                          b->stream));
  }
  return MBIS_OK;
}

mbis_status capture(mbis_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  B_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const mbis_status st = enqueue_step(b);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st != MBIS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  B_TRY(e);
  b->graph = g;
  B_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return MBIS_OK;
}

mbis_status check_ctx(const mbis_ctx* c) {
  if (!c || !c->has_metric) return berr(MBIS_E_STATE, "mbis_batch: every context needs a metric");
  if (c->opts.precision != MBIS_MIXED || c->tables_mode != 1 || (c->opts.marg & MBIS_MARG_TIME))
    return berr(MBIS_E_UNSUPPORTED,
                "mbis_batch: contexts must be mixed precision with fixed extrinsics and phase "
                "(or phase + distance) marginalisation");
  if (c->rb_use) return berr(MBIS_E_UNSUPPORTED, "mbis_batch: a context evaluates relative binning (mbis_rb_use)");
  return MBIS_OK;
}

// A context re-targeted since the launch arguments were made (mbis_set_metric rebuilds its
// tables, mbis_set_proposal moves the Gaussian): rebuild the arguments and re-capture.
mbis_status refresh(mbis_batch* b) {
  bool stale = false;
  for (int i = 0; i < b->n; ++i) stale |= b->ctx[i]->gen != b->gen[i];
  if (!stale) return MBIS_OK;
  for (int i = 0; i < b->n; ++i)
    if (const mbis_status st = check_ctx(b->ctx[i]); st != MBIS_OK) return st;
  B_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n; ++i) {
    // a re-targeted prior box may begin or stop reaching cuts inside the grid
    const bool want = b->ctx[i]->may_cut && b->ns[i] >= kOrderMinSamples;
    if (want && !b->perm[i]) {
      B_TRY(cudaMalloc(&b->perm[i], sizeof(int32_t) * b->ns[i]));
      B_TRY(cudaMalloc(&b->hist[i], sizeof(int32_t) * order_keys(b->ctx[i]->n_bins, kFoldOrderGran)));
    } else if (!want && b->perm[i]) {
      cudaFree(b->perm[i]);
      cudaFree(b->hist[i]);
      b->perm[i] = b->hist[i] = nullptr;
    }
    b->hargs[i] = batch_args(b, i);
  }
  B_TRY(cudaMemcpy(b->d_args, b->hargs.data(), sizeof(LikeArgs) * b->n, cudaMemcpyHostToDevice));
  for (int i = 0; i < b->n; ++i) b->gen[i] = b->ctx[i]->gen;
  if (const mbis_status st = build_items(b); st != MBIS_OK) return st;
  return capture(b);
}

}  // namespace

extern "C" {

mbis_status mbis_batch_create(int32_t n_ctx, mbis_ctx* const* ctxs, const int64_t* n_samples, const uint64_t* seeds,
                              mbis_batch** out) {
  if (out) *out = nullptr;
  if (n_ctx < 1 || !ctxs || !n_samples || !seeds || !out) return berr(MBIS_E_INVALID, "mbis_batch_create: bad argument");
  for (int i = 0; i < n_ctx; ++i) {
    if (const mbis_status st = check_ctx(ctxs[i]); st != MBIS_OK) return st;
    if (n_samples[i] < 1 || n_samples[i] > ((int64_t)1 << 30))
      return berr(MBIS_E_INVALID, "mbis_batch_create: n_samples must be in [1, 2^30]");
  }
  mbis_batch* b = new (std::nothrow) mbis_batch();
  if (!b) return berr(MBIS_E_OOM, "mbis_batch_create: host allocation failed");
  b->n = n_ctx;
  b->ctx.assign(ctxs, ctxs + n_ctx);
  for (int i = 0; i < n_ctx; ++i) b->gen.push_back(ctxs[i]->gen);
  b->ns.assign(n_samples, n_samples + n_ctx);
  b->seeds.assign(seeds, seeds + n_ctx);
  b->theta.assign(n_ctx, nullptr);
  b->logq.assign(n_ctx, nullptr);
  b->logp.assign(n_ctx, nullptr);
  b->ll.assign(n_ctx, nullptr);
  b->perm.assign(n_ctx, nullptr);
  b->hist.assign(n_ctx, nullptr);
  b->hargs.assign(n_ctx, LikeArgs{});
  auto fail = [&](mbis_status st) {
    mbis_batch_destroy(b);
    return st;
  };
#define C_TRY(call)                                                                               \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      berr(e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,                            \
           std::string("mbis_batch_create: ") + #call + ": " + cudaGetErrorString(e_));           \
      return fail(e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA);                     \
    }                                                                                             \
  } while (0)
  C_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  int64_t total_tiles = 0;
  for (int i = 0; i < n_ctx; ++i) {
    const mbis_ctx* c = ctxs[i];
    const int64_t n = n_samples[i];
    C_TRY(cudaMalloc(&b->theta[i], sizeof(double) * n * c->P));
    C_TRY(cudaMalloc(&b->logq[i], sizeof(double) * n));
    C_TRY(cudaMalloc(&b->logp[i], sizeof(double) * n));
    C_TRY(cudaMalloc(&b->ll[i], sizeof(double) * n));
    if (c->may_cut && n >= kOrderMinSamples) {
      C_TRY(cudaMalloc(&b->perm[i], sizeof(int32_t) * n));
      C_TRY(cudaMalloc(&b->hist[i], sizeof(int32_t) * order_keys(c->n_bins, kFoldOrderGran)));
    }
    b->hargs[i] = batch_args(b, i);
    total_tiles += (n + 63) / 64;  // the work list at the smallest tile the autotuner tries
  }
  if (total_tiles > INT32_MAX) {
    berr(MBIS_E_INVALID, "mbis_batch_create: more than 2^31 sample tiles");
    return fail(MBIS_E_INVALID);
  }
  b->items_cap = total_tiles;
  C_TRY(cudaMalloc(&b->d_args, sizeof(LikeArgs) * n_ctx));
  C_TRY(cudaMemcpy(b->d_args, b->hargs.data(), sizeof(LikeArgs) * n_ctx, cudaMemcpyHostToDevice));
  C_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)b->items_cap));
  C_TRY(cudaMalloc(&b->d_next, 2 * sizeof(int32_t)));
  C_TRY(cudaMalloc(&b->d_ctr, sizeof(uint64_t) * n_ctx));
  C_TRY(cudaMallocHost(&b->h_ctr, sizeof(uint64_t) * n_ctx));
  C_TRY(cudaMallocHost(&b->h_res, sizeof(double) * 4 * n_ctx));
  std::memset(b->h_ctr, 0, sizeof(uint64_t) * n_ctx);
#undef C_TRY
  mbis_status st = build_items(b);
  if (st != MBIS_OK) return fail(st);
  st = capture(b);
  if (st != MBIS_OK) return fail(st);
  *out = b;
  return MBIS_OK;
}

void mbis_batch_destroy(mbis_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int i = 0; i < b->n; ++i) {
    if (b->theta[i]) cudaFree(b->theta[i]);
    if (b->logq[i]) cudaFree(b->logq[i]);
    if (b->logp[i]) cudaFree(b->logp[i]);
    if (b->ll[i]) cudaFree(b->ll[i]);
    if (b->perm[i]) cudaFree(b->perm[i]);
    if (b->hist[i]) cudaFree(b->hist[i]);
  }
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_next) cudaFree(b->d_next);
  if (b->d_ctr) cudaFree(b->d_ctr);
  if (b->h_ctr) cudaFreeHost(b->h_ctr);
  if (b->h_res) cudaFreeHost(b->h_res);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

mbis_status mbis_batch_step(mbis_batch* b, uint64_t step, mbis_summary* out) {
  if (!b || !out) return berr(MBIS_E_INVALID, "mbis_batch_step: null argument");
  if (const mbis_status st = refresh(b); st != MBIS_OK) return st;
  for (int i = 0; i < b->n; ++i) b->h_ctr[i] = step * (uint64_t)b->ns[i];
  B_TRY(cudaGraphLaunch(b->exec, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n; ++i) {
    const double* r = b->h_res + 4 * i;
    const double m = r[0], s1 = r[1], s2 = r[2];
    out[i].max_logw = m;
    out[i].s1 = s1;
    out[i].s2 = s2;
    out[i].n = b->ns[i];
    out[i].all_zero = !(m > -INFINITY) || !(s1 > 0.0);
    out[i].ess = s2 > 0.0 ? s1 * s1 / s2 : 0.0;
    out[i].log_z = (m > -INFINITY && s1 > 0.0) ? m + log(s1) - log((double)b->ns[i]) : -INFINITY;
  }
  return MBIS_OK;
}

mbis_status mbis_batch_loglike(mbis_batch* b, void* stream) {
  if (!b) return berr(MBIS_E_INVALID, "mbis_batch_loglike: null batch");
  if (const mbis_status st = refresh(b); st != MBIS_OK) return st;
  B_TRY(launch_items(b, static_cast<cudaStream_t>(stream)));
  return MBIS_OK;
}

mbis_status mbis_batch_buffers(mbis_batch* b, int32_t i, double** theta, double** loglike) {
  if (!b || i < 0 || i >= b->n) return berr(MBIS_E_INVALID, "mbis_batch_buffers: bad index");
  if (theta) *theta = b->theta[i];
  if (loglike) *loglike = b->ll[i];
  return MBIS_OK;
}

mbis_status mbis_batch_copy_out(mbis_batch* b, int32_t i, double* theta_host, double* loglike_host) {
  if (!b || i < 0 || i >= b->n) return berr(MBIS_E_INVALID, "mbis_batch_copy_out: bad index");
  B_TRY(cudaStreamSynchronize(b->stream));
  if (theta_host)
    B_TRY(cudaMemcpy(theta_host, b->theta[i], sizeof(double) * b->ns[i] * b->ctx[i]->P, cudaMemcpyDeviceToHost));
  if (loglike_host) B_TRY(cudaMemcpy(loglike_host, b->ll[i], sizeof(double) * b->ns[i], cudaMemcpyDeviceToHost));
  return MBIS_OK;
}

mbis_status mbis_batch_autotune(mbis_batch* b, int32_t* grid_out, float* ms_out) {
  if (!b) return berr(MBIS_E_INVALID, "mbis_batch_autotune: null batch");
  if (const mbis_status st = refresh(b); st != MBIS_OK) return st;
  // fill the sample buffers once (and their sample order)
  for (int i = 0; i < b->n; ++i) b->h_ctr[i] = 0;
  B_TRY(cudaGraphLaunch(b->exec, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  B_TRY(cudaEventCreate(&e0));
  B_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_grid = sms * kBatchCtasPerSm, best_tile = kMixedThreads;
  // the tile shape (samples per CTA) and the persistent grid (CTAs per SM, up to what the
  // shape's registers and shared memory allow)
  for (const int tile : {64, kMixedThreads, 256}) {
    b->tile = tile;
    if (const mbis_status st = build_items(b); st != MBIS_OK) return st;
    const int cmax = batch_ctas_per_sm(tile);
    for (const int c : {cmax / 2, (3 * cmax) / 4, cmax}) {
      if (c < 1) continue;
      b->grid = sms * c;
      float t = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        B_TRY(cudaEventRecord(e0, b->stream));
        B_TRY(launch_items(b, b->stream));
        B_TRY(cudaEventRecord(e1, b->stream));
        B_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t += ms;  // first repetition warms up
      }
      if (t < best) {
        best = t;
        best_grid = b->grid;
        best_tile = tile;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tile = best_tile;
  b->grid = best_grid;
  if (const mbis_status st = build_items(b); st != MBIS_OK) return st;
  if (grid_out) *grid_out = best_grid;
  if (ms_out) *ms_out = best / 2.0f;
  return capture(b);
}

mbis_status mbis_batch_set_shape(mbis_batch* b, int32_t samples_per_cta, int32_t ctas_per_sm) {
  if (!b) return berr(MBIS_E_INVALID, "mbis_batch_set_shape: null batch");
  if (samples_per_cta != 64 && samples_per_cta != kMixedThreads && samples_per_cta != 256)
    return berr(MBIS_E_INVALID, "mbis_batch_set_shape: samples per CTA must be 64, 128 or 256");
  if (ctas_per_sm < 1 || ctas_per_sm > batch_ctas_per_sm(samples_per_cta))
    return berr(MBIS_E_INVALID, "mbis_batch_set_shape: CTAs per SM out of range for this tile");
  if (const mbis_status st = refresh(b); st != MBIS_OK) return st;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  B_TRY(cudaStreamSynchronize(b->stream));
  b->tile = samples_per_cta;
  b->grid = sms * ctas_per_sm;
  if (const mbis_status st = build_items(b); st != MBIS_OK) return st;
  return capture(b);
}

mbis_status mbis_batch_shape(const mbis_batch* b, int32_t* samples_per_cta, int32_t* grid) {
  if (!b) return berr(MBIS_E_INVALID, "mbis_batch_shape: null batch");
  if (samples_per_cta) *samples_per_cta = b->tile;
  if (grid) *grid = b->grid;
  return MBIS_OK;
}

}  // extern "C"
