// server.cpp -- served stream of parameter-estimation requests (continuous admission).
//
// A worker thread owns every device call of the server.  Requests wait in a FIFO queue
// until a slot is free and their device footprint fits under the cap beside the requests
// already admitted.  An admitted request gets a slot: its own non-blocking stream, a
// completion event and pinned host scratch; its context is created on that stream with
// stream-ordered allocations from the server's memory pool, so admitting a request never
// synchronises the device.  The worker then drives each request's ESS-target loop one
// batch at a time (issue on the slot's stream, poll its event, read the batch summary,
// issue the next), so batches of different requests overlap on the GPU, and a slot that
// finishes is refilled from the queue at once.  The arithmetic of a request is the ESS
// state machine that mbis_run_to_ess runs, on the request's own context and Philox key,
// so its result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace mbis;

namespace {

struct Request {
  uint64_t id = 0;
  mbis_request r = {};
  std::vector<unsigned char> strain;
  std::vector<double> psd, mean, chol, lo, hi, rb_fiducial;
  std::vector<mbis_detector> dets;
  std::vector<int32_t> ids;
  int64_t footprint = 0;
  double t_submit = 0.0, t_admit = 0.0;
};

struct ServerSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double* h_scratch = nullptr;  // pinned, kHostScratch doubles
  std::unique_ptr<Request> req;
  mbis_ctx* ctx = nullptr;
  EssBuffers buf = {};
  EssState st;
  bool busy = false;
};

}  // namespace

struct mbis_server {
  mbis_server_options o = {};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::map<uint64_t, mbis_result> finished;
  std::deque<uint64_t> finished_order;
  std::set<uint64_t> pending;  // submitted and not yet finished
  std::vector<ServerSlot> slots;
  cudaMemPool_t pool = nullptr;
  std::thread worker;
  bool stop = false;
  mbis_server_stats stats = {};
  uint64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

mbis_status serr(mbis_status st, const std::string& m) {
  set_last_error(m);
  return st;
}

bool is_fold(const std::vector<int32_t>& ids) {
  for (int32_t id : ids)
    if (id == kRa || id == kDec || id == kPsi || id == kIota) return false;
  return true;
}

size_t round_alloc(size_t b) { return (b + 511) / 512 * 512; }

int64_t request_footprint(const Request& q) {
  const mbis_request& r = q.r;
  size_t t = ctx_footprint_bytes(r.event.n_det, r.grid.n_bins, r.event.dtype, r.opts, is_fold(q.ids));
  t += round_alloc(sizeof(double) * (size_t)r.ess.batch * r.P) + 4 * round_alloc(sizeof(double) * (size_t)r.ess.batch);
  if (r.opts.precision == MBIS_MIXED && !(r.opts.marg & MBIS_MARG_TIME) && is_fold(q.ids)) {
    // scratch of a split folded launch: per-part sums, amplitude and cut per sample
    const size_t parts = ((size_t)r.grid.n_bins + kPartBins - 1) / kPartBins, nb = (size_t)r.ess.batch;
    t += round_alloc(16 * parts * nb) + round_alloc(8 * nb) + round_alloc(4 * nb);
  }
  if (r.opts.precision == MBIS_MIXED) {
    // sample order of a launch: the permutation and the key counts
    t += round_alloc(4 * (size_t)r.ess.batch) + round_alloc(4 * (size_t)order_keys(r.grid.n_bins, kFoldOrderGran));
  }
  if (r.rb_fiducial) {
    // relative binning: prefix tables, their build scratch, edge records, weights, edges
    const size_t n = (size_t)r.grid.n_bins, nb = (size_t)r.rb_max_bins;
    t += round_alloc(32 * (n + 1)) + round_alloc(32 * n) + round_alloc(48 * (nb + 1)) + round_alloc(8 * nb) +
         round_alloc(4 * (nb + 1));
  }
  return (int64_t)t;
}

template <typename T>
cudaError_t palloc(mbis_server* s, ServerSlot& sl, T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = cudaMallocFromPoolAsync(&q, bytes, s->pool, sl.stream);
  if (e == cudaSuccess) *p = static_cast<T*>(q);
  return e;
}

void pfree(ServerSlot& sl, double*& p) {
  if (p) cudaFreeAsync(p, sl.stream);
  p = nullptr;
}

// release a slot's resources and publish the request's result
void finish(mbis_server* s, ServerSlot& sl, mbis_status status, const std::string& msg) {
  mbis_result res = {};
  Request& q = *sl.req;
  res.id = q.id;
  res.tag = q.r.tag;
  res.status = status;
  ess_result(sl.st, &res.summary, &res.n_drawn, &res.n_used);
  res.t_submit = q.t_submit;
  res.t_admit = q.t_admit;
  res.footprint_bytes = q.footprint;
  std::snprintf(res.message, sizeof(res.message), "%s", msg.c_str());
  if (sl.ctx) mbis_destroy(sl.ctx);  // stream-ordered frees on the slot's stream
  sl.ctx = nullptr;
  pfree(sl, sl.buf.theta);
  pfree(sl, sl.buf.log_q);
  pfree(sl, sl.buf.log_prior);
  pfree(sl, sl.buf.loglike);
  pfree(sl, sl.buf.weights);
  cudaStreamSynchronize(sl.stream);  // the memory is back in the pool before it is accounted free
  res.t_done = s->now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.bytes_in_use -= q.footprint;
    s->stats.active -= 1;
    if (status == MBIS_OK)
      s->stats.completed += 1;
    else
      s->stats.failed += 1;
    s->pending.erase(q.id);
    s->finished[q.id] = res;
    s->finished_order.push_back(q.id);
  }
  s->cv_done.notify_all();
  sl.req.reset();
  sl.st = EssState{};
  sl.busy = false;
}

std::string ctx_message(const mbis_ctx* c) {
  const char* m = mbis_last_error(c);
  return m ? std::string(m) : std::string();
}

// create the request's context and buffers on the slot's stream and issue its first batch
void start(mbis_server* s, ServerSlot& sl) {
  Request& q = *sl.req;
  const mbis_request& r = q.r;
  CtxEnv env;
  env.stream = sl.stream;
  env.pool = s->pool;
  env.h_scratch = sl.h_scratch;
  mbis_status st = create_ctx(&r.event, r.psd, r.dets, &r.grid, &r.opts, env, &sl.ctx);
  if (st != MBIS_OK) return finish(s, sl, st, ctx_message(nullptr));
  st = mbis_set_metric(sl.ctx, r.P, r.ids, r.mean, r.chol, r.scale, r.lo, r.hi, r.prior_flags);
  if (st != MBIS_OK) return finish(s, sl, st, ctx_message(sl.ctx));
  if (r.rb_fiducial) {
    std::vector<int32_t> edges((size_t)r.rb_max_bins + 1);
    int32_t n_rb = 0;
    st = mbis_rb_edges(sl.ctx, r.rb_fiducial, r.rb_n_sigma, r.rb_eps_rad, r.rb_max_bins, edges.data(), &n_rb);
    if (st == MBIS_OK) st = mbis_rb_setup(sl.ctx, r.rb_fiducial, n_rb, edges.data());
    if (st == MBIS_OK) st = mbis_rb_use(sl.ctx, 1);
    if (st != MBIS_OK) return finish(s, sl, st, ctx_message(sl.ctx));
  }
  const size_t nb = (size_t)r.ess.batch;
  cudaError_t e = palloc(s, sl, &sl.buf.theta, sizeof(double) * nb * r.P);
  if (e == cudaSuccess) e = palloc(s, sl, &sl.buf.log_q, sizeof(double) * nb);
  if (e == cudaSuccess) e = palloc(s, sl, &sl.buf.log_prior, sizeof(double) * nb);
  if (e == cudaSuccess) e = palloc(s, sl, &sl.buf.loglike, sizeof(double) * nb);
  if (e == cudaSuccess) e = palloc(s, sl, &sl.buf.weights, sizeof(double) * nb);
  if (e != cudaSuccess)
    return finish(s, sl, e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
                  std::string("request buffers: ") + cudaGetErrorString(e));
  st = ess_begin(sl.ctx, &r.ess, &sl.st);
  if (st == MBIS_OK) st = ess_issue(sl.ctx, &sl.st, sl.buf, sl.stream);
  if (st != MBIS_OK) return finish(s, sl, st, ctx_message(sl.ctx));
  e = cudaEventRecord(sl.done, sl.stream);
  if (e != cudaSuccess) return finish(s, sl, MBIS_E_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
}

// one look at a busy slot: false when its batch is still running
bool advance(mbis_server* s, ServerSlot& sl) {
  const cudaError_t q = cudaEventQuery(sl.done);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) {
    finish(s, sl, MBIS_E_CUDA, std::string("batch: ") + cudaGetErrorString(q));
    return true;
  }
  mbis_status st = ess_complete(sl.ctx, &sl.st);
  if (st != MBIS_OK) {
    finish(s, sl, st, ctx_message(sl.ctx));
    return true;
  }
  if (sl.st.done) {
    finish(s, sl, MBIS_OK, "");
    return true;
  }
  st = ess_issue(sl.ctx, &sl.st, sl.buf, sl.stream);
  if (st != MBIS_OK) {
    finish(s, sl, st, ctx_message(sl.ctx));
    return true;
  }
  const cudaError_t e = cudaEventRecord(sl.done, sl.stream);
  if (e != cudaSuccess) finish(s, sl, MBIS_E_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
  return true;
}

void worker_main(mbis_server* s) {
  cudaSetDevice(s->o.device);
  for (;;) {
    std::vector<int> admitted;
    bool any_busy = false, cancel = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stats.active == 0 && s->queue.empty() && !s->stop)
        s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) {
        s->stats.queued -= (int64_t)s->queue.size();
        for (const auto& q : s->queue) s->pending.erase(q->id);
        s->queue.clear();
        cancel = true;
      }
    }
    if (cancel) {
      // requests on the device end after their batch in flight
      for (ServerSlot& sl : s->slots)
        if (sl.busy) {
          cudaEventSynchronize(sl.done);
          finish(s, sl, MBIS_E_STATE, "cancelled: the server was destroyed");
        }
      break;
    }
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // first in, first out: the head waits for memory rather than being overtaken
      while (!s->queue.empty()) {
        int free_slot = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
          if (!s->slots[i].busy) {
            free_slot = (int)i;
            break;
          }
        if (free_slot < 0) break;
        if (s->stats.bytes_in_use + s->queue.front()->footprint > s->o.hbm_cap_bytes) break;
        ServerSlot& sl = s->slots[free_slot];
        sl.req = std::move(s->queue.front());
        s->queue.pop_front();
        sl.busy = true;
        sl.req->t_admit = s->now();
        s->stats.queued -= 1;
        s->stats.active += 1;
        s->stats.bytes_in_use += sl.req->footprint;
        s->stats.bytes_peak = std::max(s->stats.bytes_peak, s->stats.bytes_in_use);
        s->stats.max_active_seen = std::max<int32_t>(s->stats.max_active_seen, (int32_t)s->stats.active);
        admitted.push_back(free_slot);
      }
    }
    for (int i : admitted) start(s, s->slots[i]);
    bool progressed = !admitted.empty();
    for (ServerSlot& sl : s->slots)
      if (sl.busy) {
        any_busy = true;
        progressed |= advance(s, sl);
      }
    if (!progressed && any_busy) {
      // nothing finished: wait briefly, or until a submission arrives
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

bool copy_request(const mbis_request* r, Request* q, std::string* why) {
  const mbis_event& ev = r->event;
  if (!ev.strain || !r->psd || !r->dets || !r->ids || !r->mean || !r->chol || !r->lo || !r->hi) {
    *why = "null array";
    return false;
  }
  if (ev.n_det < 1 || ev.n_det > kMaxDet || r->grid.n_bins < 1 || r->P < 1 || r->P > kMaxP ||
      (ev.dtype != MBIS_C128 && ev.dtype != MBIS_C64)) {
    *why = "n_det must be 1..4, n_bins >= 1, P 1..11, dtype C128 or C64";
    return false;
  }
  if (r->ess.batch < 1 || r->ess.max_samples < 1) {
    *why = "ess.batch and ess.max_samples must be >= 1";
    return false;
  }
  if (r->rb_fiducial && (!(r->rb_n_sigma > 0.0) || !(r->rb_eps_rad > 0.0) || r->rb_max_bins < 1 ||
                         r->rb_max_bins > r->grid.n_bins)) {
    *why = "relative binning needs rb_n_sigma > 0, rb_eps_rad > 0 and 1 <= rb_max_bins <= n_bins";
    return false;
  }
  const size_t nb = (size_t)ev.n_det * r->grid.n_bins, P = (size_t)r->P;
  const size_t csz = ev.dtype == MBIS_C128 ? 16 : 8;
  q->r = *r;
  q->strain.assign((const unsigned char*)ev.strain, (const unsigned char*)ev.strain + csz * nb);
  q->psd.assign(r->psd, r->psd + nb);
  q->dets.assign(r->dets, r->dets + ev.n_det);
  q->ids.assign(r->ids, r->ids + P);
  q->mean.assign(r->mean, r->mean + P);
  q->chol.assign(r->chol, r->chol + P * P);
  q->lo.assign(r->lo, r->lo + P);
  q->hi.assign(r->hi, r->hi + P);
  q->r.event.strain = q->strain.data();
  q->r.psd = q->psd.data();
  q->r.dets = q->dets.data();
  q->r.ids = q->ids.data();
  q->r.mean = q->mean.data();
  q->r.chol = q->chol.data();
  q->r.lo = q->lo.data();
  q->r.hi = q->hi.data();
  if (r->rb_fiducial) {
    q->rb_fiducial.assign(r->rb_fiducial, r->rb_fiducial + kNumSlots);
    q->r.rb_fiducial = q->rb_fiducial.data();
  }
  return true;
}

void release_slots(mbis_server* s) {
  for (ServerSlot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.h_scratch) cudaFreeHost(sl.h_scratch);
    sl = ServerSlot{};
  }
}

}  // namespace

extern "C" {

mbis_status mbis_server_create(const mbis_server_options* o, mbis_server** out) {
  if (out) *out = nullptr;
  if (!o || !out) return serr(MBIS_E_INVALID, "mbis_server_create: null argument");
  if (o->max_active < 1 || o->max_active > 256 || o->hbm_cap_bytes < 1)
    return serr(MBIS_E_INVALID, "mbis_server_create: max_active must be 1..256 and hbm_cap_bytes > 0");
  mbis_server* s = new (std::nothrow) mbis_server();
  if (!s) return serr(MBIS_E_OOM, "mbis_server_create: host allocation failed");
  s->o = *o;
  s->t0 = std::chrono::steady_clock::now();
  s->stats.bytes_cap = o->hbm_cap_bytes;
  cudaError_t e = cudaSetDevice(o->device);
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = o->device;
  if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // keep freed memory in the pool for the next request
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  s->slots.resize(o->max_active);
  for (ServerSlot& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_scratch, sizeof(double) * kHostScratch);
  }
  if (e != cudaSuccess) {
    release_slots(s);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return serr(e == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,
                std::string("mbis_server_create: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return MBIS_OK;
}

mbis_status mbis_server_submit(mbis_server* s, const mbis_request* r, uint64_t* id, int64_t* footprint_out) {
  if (!s || !r || !id) return serr(MBIS_E_INVALID, "mbis_server_submit: null argument");
  auto q = std::make_unique<Request>();
  std::string why;
  if (!copy_request(r, q.get(), &why)) return serr(MBIS_E_INVALID, "mbis_server_submit: " + why);
  q->footprint = request_footprint(*q);
  if (q->footprint > s->o.hbm_cap_bytes)
    return serr(MBIS_E_INVALID, "mbis_server_submit: the request's footprint (" + std::to_string(q->footprint) +
                                    " bytes) exceeds the server's cap");
  if (footprint_out) *footprint_out = q->footprint;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return serr(MBIS_E_STATE, "mbis_server_submit: the server is stopping");
    q->id = s->next_id++;
    q->t_submit = s->now();
    *id = q->id;
    s->pending.insert(q->id);
    s->queue.push_back(std::move(q));
    s->stats.submitted += 1;
    s->stats.queued += 1;
  }
  s->cv_work.notify_one();
  return MBIS_OK;
}

mbis_status mbis_server_wait(mbis_server* s, uint64_t id, double timeout_s, mbis_result* out) {
  if (!s || !out) return serr(MBIS_E_INVALID, "mbis_server_wait: null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->finished.count(id) > 0; };
  if (!ready() && !s->pending.count(id)) return serr(MBIS_E_INVALID, "mbis_server_wait: unknown request id");
  if (timeout_s < 0) {
    s->cv_done.wait(lk, [&] { return ready() || !s->pending.count(id); });
  } else {
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return ready() || !s->pending.count(id); });
  }
  if (!ready()) {
    if (!s->pending.count(id)) return serr(MBIS_E_STATE, "mbis_server_wait: the request was dropped");
    return serr(MBIS_E_TIMEOUT, "mbis_server_wait: the request is not done yet");
  }
  *out = s->finished[id];
  s->finished.erase(id);
  s->finished_order.erase(std::find(s->finished_order.begin(), s->finished_order.end(), id));
  return MBIS_OK;
}

mbis_status mbis_server_poll(mbis_server* s, mbis_result* out, int32_t max, int32_t* n_out) {
  if (!s || !n_out || (max > 0 && !out)) return serr(MBIS_E_INVALID, "mbis_server_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t n = 0;
  while (n < max && !s->finished_order.empty()) {
    const uint64_t id = s->finished_order.front();
    s->finished_order.pop_front();
    out[n++] = s->finished[id];
    s->finished.erase(id);
  }
  *n_out = n;
  return MBIS_OK;
}

mbis_status mbis_server_stats_get(mbis_server* s, mbis_server_stats* out) {
  if (!s || !out) return serr(MBIS_E_INVALID, "mbis_server_stats_get: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return MBIS_OK;
}

void mbis_server_destroy(mbis_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  s->cv_done.notify_all();
  release_slots(s);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
