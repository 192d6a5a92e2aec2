/*
 * mbis.h -- C ABI of the GB300 (sm_103a) implementation of metric-based importance
 * sampling for compact-binary parameter estimation (Nitz, "Robust, Rapid, and Simple
 * Gravitational-wave Parameter Estimation").
 *
 * One call sequence per event:
 *   mbis_create      event data, PSD, detectors, frequency grid, options -> context
 *   mbis_set_metric  Gaussian proposal in the Fisher metric + prior box
 *   mbis_draw        proposal samples theta ~ g, log g, log prior         (Eq. 5: g, pi)
 *   mbis_loglike     log L(d | theta) for every sample                    (Eqs. 1-3)
 *   mbis_reduce      weights, ESS, log evidence                           (Eqs. 5-6)
 *   mbis_destroy
 *
 * Conventions shared by every entry point:
 *   - Status codes, never exceptions or aborts.  mbis_last_error() gives the message of
 *     the last failure on a context (or of the last context-free failure when ctx is NULL).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of
 *     the current device (e.g. a torch tensor's data_ptr()).  The caller owns every buffer
 *     it passes; the library deep-copies what it keeps and never frees caller memory.
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *     device work of a call is enqueued on that stream.  Calls that return host results
 *     (mbis_reduce, mbis_fisher, mbis_inject) synchronise that stream before returning.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Parameter slots (full 11-parameter sample):
 *       0 Mc (detector-frame chirp mass, Msun)  1 q = m1/m2 (>= 1 inside the prior)
 *       2 chi1z  3 chi2z  4 RA (rad)  5 dec (rad)  6 psi (rad)  7 iota (rad)
 *       8 d_L (Mpc)  9 t_c (s, geocentre)  10 phi_c (rad, GW phase)
 *   - Sample arrays are structure-of-arrays: theta[p * n + i] is slot ids[p] of sample i.
 */
#ifndef MBIS_H
#define MBIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbis_ctx mbis_ctx;

typedef enum {
  MBIS_OK = 0,
  MBIS_E_INVALID = 1,     /* bad argument: null pointer, size, slot id, inconsistent mode */
  MBIS_E_OOM = 2,         /* device or host allocation failed */
  MBIS_E_CUDA = 3,        /* a CUDA call failed; message holds cudaGetErrorString */
  MBIS_E_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  MBIS_E_STATE = 5,       /* call out of order (e.g. mbis_draw before mbis_set_metric) */
  MBIS_E_UNSUPPORTED = 6  /* valid request this build does not implement */
} mbis_status;

enum {
  MBIS_P_MC = 0, MBIS_P_Q = 1, MBIS_P_CHI1 = 2, MBIS_P_CHI2 = 3, MBIS_P_RA = 4, MBIS_P_DEC = 5,
  MBIS_P_PSI = 6, MBIS_P_IOTA = 7, MBIS_P_DL = 8, MBIS_P_TC = 9, MBIS_P_PHIC = 10, MBIS_NPAR = 11
};

/* marginalisation bits (Sec. III: analytic phase and distance, numeric time) */
enum { MBIS_MARG_PHASE = 1, MBIS_MARG_DISTANCE = 2, MBIS_MARG_TIME = 4 };
/* strain storage (the PSD is always double: aLIGO-like values ~1e-47 lie below FLT_MIN) */
enum { MBIS_C128 = 0, MBIS_C64 = 1 };
/* arithmetic of mbis_loglike */
enum { MBIS_FP64 = 0, MBIS_MIXED = 1 };
/* prior flags */
enum { MBIS_PRIOR_M1M2 = 1 };

/* Uniform grid f_k = f_lo + k df, k = 0 .. n_bins-1 (Eq. 1 as a rectangle sum, weight df). */
typedef struct {
  double f_lo, df;
  int32_t n_bins;
} mbis_freq_grid;

/* Detector: vertex in Earth-centred Earth-fixed metres, unit arm vectors. */
typedef struct {
  double vertex_m[3], xarm[3], yarm[3];
} mbis_detector;

typedef struct {
  int32_t n_det;        /* 1..4 */
  int32_t dtype;        /* strain storage: MBIS_C128 (complex128) or MBIS_C64 (complex64) */
  const void* strain;   /* host, [n_det][n_bins] interleaved (re, im), frequency-domain data d(f) */
  double gmst_rad;      /* Greenwich mean sidereal time at the reference time */
  double fixed[11];     /* values of the slots that are neither sampled nor marginalised */
} mbis_event;

typedef struct {
  int32_t precision;    /* MBIS_FP64 or MBIS_MIXED */
  uint32_t marg;        /* 0, PHASE, PHASE|DISTANCE, or TIME */
  int32_t n_tshift;     /* TIME: number of shifts J (tau_j = (j - J/2) dt_shift) */
  double dt_shift;      /* TIME: shift spacing, s */
  double dmin_mpc, dmax_mpc;  /* DISTANCE: prior p(d) ~ d^2 on [dmin, dmax] */
} mbis_options;

/* Running reducer state and its derived summary (Eq. 6).  max_logw = -inf and ess = 0
 * when every weight is zero (all_zero = 1). */
typedef struct {
  double ess, log_z, max_logw;
  int64_t n;
  double s1, s2;        /* sum e^(log w - max), sum e^(2 (log w - max)) */
  int32_t all_zero;
} mbis_summary;

/* Create a context for one event.  Paper: Eqs. 1-3 (data d, PSD S_n).
 *   event, psd (host, [n_det][n_bins] double, one-sided, > 0), dets
 *   (host, n_det), grid, opts: read during the call and copied to the device; the caller
 *   may free them afterwards.  *out receives the context (NULL on failure).
 *   Errors: MBIS_E_INVALID (null, n_det/n_bins/grid out of range, unsupported marg or
 *   precision combination), MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_create(const mbis_event* event, const double* psd, const mbis_detector* dets,
                        const mbis_freq_grid* grid, const mbis_options* opts, mbis_ctx** out);

/* Set the proposal: a Gaussian N(mean, scale^2 L L^T) over the P sampled slots (the
 * local metric of Sec. II A, whose tiling the proposal of Sec. II approximates), and the
 * prior box.  param_ids (host, P distinct slots), mean (host, P), chol_lower (host,
 * P x P row-major lower-triangular factor, positive diagonal), prior_lo / prior_hi
 * (host, P; ignored for RA, psi, phi_c, which take their full period).  prior_flags:
 * MBIS_PRIOR_M1M2 makes the (Mc, q) prior flat in component masses (both slots must be
 * sampled).  Slots marginalised by the options may not be sampled.
 * Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_set_metric(mbis_ctx* ctx, int32_t P, const int32_t* param_ids, const double* mean,
                            const double* chol_lower, double scale, const double* prior_lo,
                            const double* prior_hi, uint32_t prior_flags);

/* Draw n proposal samples (g of Eq. 5) with Philox4x32-10: sample i uses counter
 * (lo32(ctr0+i), hi32(ctr0+i), 2, block) and key (lo32(seed), hi32(seed)); Box-Muller
 * normals z, theta = mean + scale L z, RA and phi_c wrapped into [0, 2 pi), psi into
 * [0, pi).  Outputs (device): theta [P][n] SoA, log_q [n] = unwrapped Gaussian log
 * density, log_prior [n] (-inf outside the prior).  log_q / log_prior may be NULL.
 * Errors: MBIS_E_STATE (no metric), MBIS_E_INVALID (n < 0, null theta), MBIS_E_CUDA. */
mbis_status mbis_draw(mbis_ctx* ctx, uint64_t seed, uint64_t ctr0, int64_t n, double* theta, double* log_q,
                      double* log_prior, void* cuda_stream);

/* Log likelihood ratio ln(L/L_n) of Eq. 3 (the -(d|d)/2 of Eq. 2 dropped) for n samples,
 * marginalised as the options say: PHASE -> ln I0(|Z|) - H/2; PHASE|DISTANCE ->
 * ln int p(d) I0(|Z1|/d) e^(-H1/(2 d^2)) dd; TIME -> ln mean_j e^(Re z_j - H/2).  theta
 * (device, [P][n] SoA as written by mbis_draw), loglike (device, n).  Samples with an
 * unphysical parameter (Mc <= 0, q <= 0, |chi| >= 1, d_L <= 0) get -inf.  A call with fewer
 * samples than fill the GPU shares each sample's bins among several CTAs through scratch the
 * context owns (allocated on first need, from its pool in the server), with results equal bit
 * for bit to an unsplit launch; calls on one context are therefore ordered on one stream (or
 * synchronised), like its reductions.
 * Errors: MBIS_E_STATE, MBIS_E_INVALID, MBIS_E_UNSUPPORTED, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_loglike(mbis_ctx* ctx, int64_t n, const double* theta, double* loglike, void* cuda_stream);

/* Importance weights and Kish ESS (Eqs. 5-6), evidence Z = mean(w).  Two passes on the
 * device: m = max(log L + log pi - log g), then FP64 sums S1 = sum e^(log w - m),
 * S2 = sum e^(2 (log w - m)).  Inputs (device, n each).  weights_out (device, n) gets the
 * normalised weights e^(log w - m) / S1 when not NULL.  accumulate != 0 merges this batch
 * into the context's running state and reports the merged summary; 0 reports this batch
 * alone and leaves the running state untouched.  *out (host) receives the summary;
 * the stream is synchronised.  Uses device scratch owned by the context.
 * Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_reduce(mbis_ctx* ctx, int64_t n, const double* loglike, const double* log_prior,
                        const double* log_q, double* weights_out, int32_t accumulate, mbis_summary* out,
                        void* cuda_stream);

/* mbis_reduce without a context and without any allocation.  The paper has no
 * counterpart: this is for callers that must not call cudaMalloc once they run -- e.g. a
 * low-latency loop in which an allocation would synchronise the device, or a host
 * framework that owns all device memory and forbids allocations after start-up.  The
 * caller passes the inputs (device, n each) and the outputs (weights_out: device n
 * doubles or NULL; *out: host summary of this batch); the stream is synchronised.
 * Scratch is a file-scope device array of the library (about 128 KiB on every GPU that
 * loads it, kept until exit) with room for MBIS_NOALLOC_MAX_SAMPLES samples per call;
 * larger n returns MBIS_E_INVALID with a message in mbis_last_error(NULL).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  A lookup that fails is
 * not remembered: the next call tries again.  With lazy module loading (the CUDA default)
 * that first call also loads the library's module onto the device, a one-time device
 * allocation of about 128 KiB that may synchronise: warm the entry point up once at
 * start-up (for example with n = 1) to keep it off the critical path.  All calls share the
 * array and it keeps the last call's contents; each call zeroes the part that must start
 * at zero.  Calls that overlap on the GPU (other streams or threads) race on it.
 * Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
#define MBIS_NOALLOC_MAX_SAMPLES 16777216
mbis_status mbis_reduce_noalloc(int64_t n, const double* loglike, const double* log_prior, const double* log_q,
                                double* weights_out, mbis_summary* out, void* cuda_stream);

/* Weighted mean and covariance of n proposal samples: the ingredients of refitting the
 * Gaussian proposal from importance-weighted samples (the iterative update of the proposal
 * suggested in Sec. III A).  theta (device, [P][n] as drawn), weights (device, n; e.g. the
 * normalised weights of mbis_reduce; zero or negative weights are skipped).  mean_out
 * (host, P) and cov_out (host, P x P row-major) are normalised by the sum of the weights.
 * Periodic slots (RA, phi_c: 2 pi; psi: pi) are averaged as offsets wrapped around the
 * current proposal mean.  The stream is synchronised.
 * Errors: MBIS_E_STATE (no metric), MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_weighted_moments(mbis_ctx* ctx, int64_t n, const double* theta, const double* weights,
                                  double* mean_out, double* cov_out, void* cuda_stream);

/* Replace the Gaussian proposal (mean, P x P lower Cholesky factor, scale) and keep the
 * sampled slots and prior of the last mbis_set_metric; no table is rebuilt.
 * Errors: MBIS_E_STATE, MBIS_E_INVALID. */
mbis_status mbis_set_proposal(mbis_ctx* ctx, const double* mean, const double* chol_lower, double scale);

/* The current Gaussian proposal (as set by mbis_set_metric / mbis_set_proposal, or refitted
 * by the ESS loop): mean_out (host, P), chol_out (host, P x P row-major lower), scale_out
 * (host); each may be NULL.  Errors: MBIS_E_INVALID (null context), MBIS_E_STATE (no
 * metric; reported by mbis_last_error(NULL)). */
mbis_status mbis_get_proposal(const mbis_ctx* ctx, double* mean_out, double* chol_out, double* scale_out);

typedef struct {
  double ess_target;    /* stop once the running ESS reaches this */
  int64_t batch;        /* samples per batch; the caller's buffers hold one batch */
  int64_t max_samples;  /* stop after this many draws even if the target is not reached */
  int32_t refine;       /* refit the proposal after each of the first `refine` batches */
  double refine_scale;  /* width scale of a refitted proposal (<= 0 keeps the current scale) */
  uint64_t seed;        /* Philox key; batch b uses counters [b * batch, (b + 1) * batch) */
  double refit_min_ess; /* a refit waits for this ESS: see mbis_run_to_ess (<= 0: 2P + 1) */
} mbis_ess_options;

/* ESS-target loop: batches of draw -> likelihood -> weights merged into the running state
 * until ESS >= ess_target (the paper quotes costs for a target of 10^4 effective samples,
 * App. C).  With refine > 0, each of the first `refine` batches refits the proposal
 * (weighted mean and covariance, mbis_weighted_moments) when its own ESS is at least 2P + 1;
 * batches drawn before the last refit only adapt the proposal and do not enter the
 * estimate.  With refit_min_ess above 2P + 1, a refit batch whose ESS falls short pools
 * its weighted moments with the next batches drawn from the same proposal (weights on one
 * scale) until the pooled ESS reaches refit_min_ess, or 16 batches are pooled; the refit
 * then uses the pool (if its ESS is at least 2P + 1) and counts as one of `refine`.  Buffers (device, one batch): theta [P][batch], log_q, log_prior, loglike,
 * weights [batch].  *out: summary of the estimate; n_drawn (host, nullable): every draw,
 * adaptation included; n_used (host, nullable): draws in the estimate.
 * Errors: MBIS_E_STATE, MBIS_E_INVALID, MBIS_E_UNSUPPORTED, MBIS_E_CUDA, MBIS_E_TIMEOUT. */
mbis_status mbis_run_to_ess(mbis_ctx* ctx, const mbis_ess_options* opts, double* theta, double* log_q,
                            double* log_prior, double* loglike, double* weights, mbis_summary* out,
                            int64_t* n_drawn, int64_t* n_used, void* cuda_stream);

/* ---- many events in one launch ----------------------------------------------------- */

typedef struct mbis_batch mbis_batch;

/* A batch of events whose likelihoods run in one persistent launch (one per block-entry
 * arithmetic, float-float or FP64): the 128-sample tiles of every event form a work list,
 * longest first, consumed by a persistent grid; a step
 * (draws, likelihoods, reductions, summaries of every event) is one CUDA graph replay.
 * ctxs: n_ctx contexts with a metric set, MBIS_MIXED, fixed sky/orientation, PHASE or
 * PHASE|DISTANCE marginalisation (they stay owned by the caller and must outlive the
 * batch; a context re-targeted by mbis_set_metric / mbis_set_proposal between steps is
 * picked up by the next step, which rebuilds the launch arguments and re-captures the
 * graph).  A context belongs to at most one batch at a time
 * (the batch uses the context's reduction scratch).  n_samples[i] samples per step for
 * event i (1..2^30), seeds[i] its Philox key.  The batch allocates the sample buffers of
 * every event on the device and its own non-blocking stream.
 * Errors: MBIS_E_INVALID, MBIS_E_STATE, MBIS_E_UNSUPPORTED, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_batch_create(int32_t n_ctx, mbis_ctx* const* ctxs, const int64_t* n_samples, const uint64_t* seeds,
                              mbis_batch** out);

/* One step: event i draws counters [step * n_i, (step + 1) * n_i).  out: host array of n_ctx
 * summaries (this step alone).  Synchronises the batch's own stream. */
mbis_status mbis_batch_step(mbis_batch* b, uint64_t step, mbis_summary* out);

/* Times the persistent launch on the current samples for every tile shape -- 64, 128 or 256
 * samples per CTA (the work list is rebuilt for each) -- at 1/2, 3/4 and all of the CTAs per
 * SM that the shape's registers and shared memory allow (14, 7 and 3), keeps the fastest
 * and re-captures the step graph.  Results do not depend on the shape.  grid_out / ms_out
 * (host, nullable): the chosen grid and its launch time; mbis_batch_shape reports both. */
mbis_status mbis_batch_autotune(mbis_batch* b, int32_t* grid_out, float* ms_out);

/* Sets the shape of the persistent launch instead of the autotuner: samples_per_cta (64,
 * 128 or 256) and ctas_per_sm (1 .. 14, 7 or 3 for those tiles); rebuilds the work list and
 * re-captures the step graph.  Results do not depend on the shape.
 * Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_batch_set_shape(mbis_batch* b, int32_t samples_per_cta, int32_t ctas_per_sm);

/* The current shape of the persistent launch: samples per CTA and CTAs in the grid (host,
 * nullable).  Errors: MBIS_E_INVALID. */
mbis_status mbis_batch_shape(const mbis_batch* b, int32_t* samples_per_cta, int32_t* grid);

/* The persistent likelihood launch alone, on the batch's current samples, on a caller
 * stream (for timing and tests). */
mbis_status mbis_batch_loglike(mbis_batch* b, void* cuda_stream);

/* Device pointers of event i's sample and log-likelihood buffers ([P][n_i] and [n_i]),
 * owned by the batch. */
mbis_status mbis_batch_buffers(mbis_batch* b, int32_t i, double** theta, double** loglike);

/* Copy event i's current samples (host, [P][n_i]) and log-likelihoods (host, [n_i]) out;
 * either pointer may be NULL.  Synchronises the batch's stream. */
mbis_status mbis_batch_copy_out(mbis_batch* b, int32_t i, double* theta_host, double* loglike_host);

void mbis_batch_destroy(mbis_batch* b);

/* ---- served stream: requests run to a target ESS with continuous admission ---------- */

typedef struct mbis_server mbis_server;

typedef struct {
  int64_t hbm_cap_bytes;  /* admission cap on the summed device footprint of admitted requests */
  int32_t max_active;     /* requests on the device at once (1..256); each has its own stream */
  int32_t device;         /* CUDA device the server's worker thread uses */
} mbis_server_options;

/* One parameter-estimation request: an event (as for mbis_create), its proposal (as for
 * mbis_set_metric) and the ESS-target loop options (as for mbis_run_to_ess).  Every host
 * array is deep-copied by mbis_server_submit. */
typedef struct {
  mbis_event event;
  const double* psd;          /* host, [n_det][n_bins] */
  const mbis_detector* dets;  /* host, n_det */
  mbis_freq_grid grid;
  mbis_options opts;
  int32_t P;
  const int32_t* ids;         /* host, P */
  const double* mean;         /* host, P */
  const double* chol;         /* host, P x P lower, row-major */
  double scale;
  const double* lo;           /* host, P */
  const double* hi;           /* host, P */
  uint32_t prior_flags;
  mbis_ess_options ess;
  uint64_t tag;               /* returned unchanged in the result */
  /* Optional relative binning (mbis_rb_edges / mbis_rb_setup / mbis_rb_use): when
   * rb_fiducial (host, 11 slots) is not NULL the request's ESS loop runs on the
   * relative-binning likelihood about that fiducial, with bins from mbis_rb_edges(rb_n_sigma,
   * rb_eps_rad, at most rb_max_bins).  Needs a folded, not time-marginalised context. */
  const double* rb_fiducial;
  double rb_n_sigma, rb_eps_rad;
  int32_t rb_max_bins;
} mbis_request;

typedef struct {
  uint64_t id, tag;
  int32_t status;             /* mbis_status of the request */
  int32_t pad;
  mbis_summary summary;       /* as mbis_run_to_ess */
  int64_t n_drawn, n_used;
  double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock */
  int64_t footprint_bytes;    /* device bytes reserved for the request while it ran */
  char message[160];          /* error message when status != MBIS_OK */
} mbis_result;

typedef struct {
  int64_t submitted, queued, active, completed, failed;
  int64_t bytes_in_use, bytes_peak, bytes_cap;
  int32_t max_active_seen;    /* most requests on the device at one time */
  int32_t pad;
} mbis_server_stats;

/* Not in the paper: the paper runs one event at a time.  A served stream admits requests
 * first-in first-out as soon as a slot is free and the request's device footprint fits
 * under hbm_cap_bytes beside the requests already admitted; admitted requests keep their
 * data, PSD, tables and proposal resident and run the ESS-target loop of mbis_run_to_ess
 * one batch at a time on their own streams, so the batches of different requests overlap
 * on the device.  Each request's arithmetic is that of mbis_run_to_ess on the same inputs:
 * its result does not depend on what else runs.  A background thread does the work.
 * Errors: MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_server_create(const mbis_server_options* opts, mbis_server** out);

/* Queue a request (returns at once).  *id (host) identifies its result.  A request whose
 * footprint alone exceeds hbm_cap_bytes, or that mbis_create / mbis_set_metric would
 * reject, fails here with MBIS_E_INVALID.  *footprint_out (host, nullable): the bytes the
 * request reserves. */
mbis_status mbis_server_submit(mbis_server* s, const mbis_request* req, uint64_t* id, int64_t* footprint_out);

/* Wait up to timeout_s seconds (< 0: forever) for request id; on success *out holds its
 * result and the server forgets it.  MBIS_E_TIMEOUT when it is not done in time,
 * MBIS_E_INVALID for an unknown id. */
mbis_status mbis_server_wait(mbis_server* s, uint64_t id, double timeout_s, mbis_result* out);

/* Up to max finished results not yet taken, oldest first; *n_out how many were written. */
mbis_status mbis_server_poll(mbis_server* s, mbis_result* out, int32_t max, int32_t* n_out);

mbis_status mbis_server_stats_get(mbis_server* s, mbis_server_stats* out);

/* Requests still queued are dropped; those on the device finish their batch in flight and
 * are released; then the worker stops and every resource is freed. */
void mbis_server_destroy(mbis_server* s);

/* ---- tiled proposal: template bank, prior-volume tiles, mixture draws --------------- */

typedef struct mbis_tiling mbis_tiling;

/* The sampled space of the tiled proposal (App. A): a chirp-mass coordinate x in
 * [x_lo, x_hi), mapped to the chirp mass mc_base + mod(x, mc_period) (the "cyclic chirp
 * mass"; mc_period <= 0 maps x to itself), and a mass ratio q in [q_lo, q_hi] that may
 * extend below 1 (q and 1/q name the same binary); aligned spins fixed at chi1, chi2.  The
 * prior of the space is uniform in (x, q). */
typedef struct {
  double x_lo, x_hi;
  double mc_period, mc_base;
  double q_lo, q_hi;
  double chi1, chi2;
} mbis_tiling_space;

/* Sec. II, App. A: the paper tiles the space of waveforms with a template bank and maps
 * every prior sample to the tile of its best-matching template; the match is the overlap
 * of Eq. 1's inner product between unit-norm waveforms, maximised over phase at a common
 * coalescence time (the TaylorF2 waveform of the likelihood, zero at and above the ISCO),
 * weighted by one PSD.  grid: the frequency grid; psd (host, n_bins doubles > 0 on the
 * bins the space reaches).  Every point of the space must have a live bin (an ISCO above
 * f_lo).  Copies what it needs to the device; the caller keeps ownership of its arrays.
 * Errors: MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_tiling_create(const mbis_freq_grid* grid, const double* psd, const mbis_tiling_space* space,
                               mbis_tiling** out);

/* Stochastic template placement (App. A, "Template bank generation"): the candidates
 * (host, [2][n_cand]: x row then q row, inside the space) are visited in order, and one
 * joins the bank when its match with every template already in the bank is below
 * min_match (0 < min_match < 1).  Placement stops after stop_after consecutive
 * rejections, at max_templates (1..16384) or at the end of the candidates.  Matches are
 * FP64 on the device; the accept decisions are taken on the host in candidate order.
 * Replaces any earlier bank (and drops the pool and mixture).  n_templates, n_used (host,
 * nullable): the bank size and the candidates visited.
 * Errors: MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_tiling_bank(mbis_tiling* t, int64_t n_cand, const double* cand, double min_match,
                             int64_t stop_after, int32_t max_templates, int32_t* n_templates, int64_t* n_used);

/* The bank: *n_templates (host); coords (host, nullable, [2][T]) the templates' (x, q);
 * physical (host, nullable, [2][T]) their chirp mass and mass ratio >= 1; cand_index
 * (host, nullable, [T]) their positions in the candidate list.  MBIS_E_STATE without a
 * bank. */
mbis_status mbis_tiling_templates(const mbis_tiling* t, int32_t* n_templates, double* coords, double* physical,
                                  int32_t* cand_index);

/* FP64 match of n point pairs (device, [2][n] each: x row then q row); out (device, n).
 * The matches that drive template placement.  Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_tiling_match(mbis_tiling* t, int64_t n, const double* a, const double* b, double* out,
                              void* cuda_stream);

/* Tile of each point (App. A, "Tiling the prior volume"): the template of highest match,
 * equal FP32 matches going to the template the contraction visits first (templates are
 * visited in order of live-bin count).  pts (device, [2][n]); tile (device, n int32; -1 for
 * a point outside the space); match (device, n float, nullable) the best match.  The
 * sample-by-template overlaps are one FP16 tensor-core contraction (tcgen05, FP32
 * accumulation) over the live bins, the sample waveforms computed in registers and never
 * stored; matches carry ~1e-4 absolute error at most, so points whose two best templates
 * match within that may land in either tile.  Points are processed in order of their
 * live-bin count (a device-side sort into scratch that the tiling object keeps and grows
 * to the largest n seen), so calls on one tiling object must not overlap.  Asynchronous: a
 * device-side wait that timed out is reported by the next mbis_tiling_set_pool.  Needs a
 * bank; 0 <= n < 2^31.  Errors: MBIS_E_STATE, MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_tiling_assign(mbis_tiling* t, int64_t n, const double* pts, int32_t* tile, float* match,
                               void* cuda_stream);

/* The prior sample that defines the tiles' prior volumes: pts (device, [2][n], points drawn
 * from the prior, 1 <= n < 2^31) is copied, assigned, and sorted into per-tile lists (in
 * increasing sample order).  Drops an earlier mixture.  Synchronises the stream.
 * Errors: MBIS_E_STATE, MBIS_E_INVALID (a point outside the space), MBIS_E_OOM,
 * MBIS_E_CUDA, MBIS_E_TIMEOUT. */
mbis_status mbis_tiling_set_pool(mbis_tiling* t, int64_t n, const double* pts, void* cuda_stream);

/* Pool members of every tile: counts (host, [T] int64); tile_of (device, nullable, [n]
 * int32) the pool's tile indices; members (device, nullable, [n] int32) the pool indices
 * grouped by tile, each tile in increasing order, tiles in order. */
mbis_status mbis_tiling_pool(const mbis_tiling* t, int64_t* counts, int32_t* tile_of, int32_t* members,
                             void* cuda_stream);

/* The mixture (Sec. II; App. A, "Generation of the posterior distribution"): tile j is
 * drawn with probability p_j proportional to n_j L_j, n_j its pool members (its share of
 * the prior volume) and ln L_j = loglike_tpl[j] (device, [T]) the log-likelihood ratio at
 * its template, e.g. from mbis_loglike on the templates' physical coordinates.
 * Synchronises the stream.  Errors: MBIS_E_STATE (no pool), MBIS_E_INVALID (no tile with
 * members has a finite log-likelihood), MBIS_E_CUDA. */
mbis_status mbis_tiling_set_loglike(mbis_tiling* t, const double* loglike_tpl, void* cuda_stream);

/* n draws of the mixture: draw i uses the Philox4x32-10 block of counter
 * (lo32(ctr0 + i), hi32(ctr0 + i), 3, 0) and key (lo32(seed), hi32(seed)); words 0-1 pick
 * the tile by its cumulative weight, words 2-3 one of its members by multiply-shift.
 * coords (device, nullable, [2][n]): the drawn (x, q); theta (device, [2][n]): their chirp
 * mass and mass ratio >= 1, the rows of a likelihood context sampling (Mc, q); log_q
 * (device, n): ln g = ln pi + ln p_j - ln(n_j / N); log_prior (device, n): ln pi, uniform
 * in (x, q); pool_index (device, nullable, n int32).  Errors: MBIS_E_STATE (no mixture),
 * MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_tiling_draw(mbis_tiling* t, uint64_t seed, uint64_t ctr0, int64_t n, double* coords, double* theta,
                             double* log_q, double* log_prior, int32_t* pool_index, void* cuda_stream);

void mbis_tiling_destroy(mbis_tiling* t);
const char* mbis_tiling_last_error(const mbis_tiling* t);

/* ---- P-P self-consistency (Sec. III A) --------------------------------------------- */

/* Credible level of a reference point under weighted samples: for each slot p < P,
 *   level[p] = (sum_i w_i [theta[p][i] < ref[p]] + 1/2 sum_i w_i [theta[p][i] == ref[p]]) / sum_i w_i
 * over the positive weights.  The paper validates its posteriors by the distribution of
 * this level of the true parameters over a simulated population (uniform when the method
 * is self-consistent).  theta (device, [P][n]), weights (device, n; any positive scale,
 * e.g. the normalised weights of mbis_reduce), ref (host, P), levels (device, P; NaN when
 * no weight is positive).  n >= 1, 1 <= P <= 16.  Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_credible_levels(int64_t n, int32_t P, const double* theta, const double* weights, const double* ref,
                                 double* levels, void* cuda_stream);

/* ---- relative binning (a faster approximate likelihood) ---------------------------- */

/* The paper notes (Sec. IV) that faster likelihood evaluations plug into its method
 * directly; relative binning (Zackay, Dai & Venumadhav 2018) is one.  About a fiducial
 * theta0 (host, 11 slots) the template's ratio to the fiducial is taken as linear inside each
 * of n_rb coarse bins with edges (host, n_rb + 1 increasing bin indices, edges[0] = 0,
 * edges[n_rb] = n_bins; the last edge is the frequency one past the grid), so a likelihood
 * costs n_rb + 1 phase evaluations instead of n_bins; <h|h> stays exact.  Needs a context
 * with a metric, fixed sky and orientation (the folded table) and no time marginalisation;
 * mbis_set_metric drops the set-up (a proposal refit keeps it).  Allocates its summary data
 * from the context's allocator (stream-ordered from the server's pool for a served request).
 * Errors: MBIS_E_STATE, MBIS_E_UNSUPPORTED, MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_rb_setup(mbis_ctx* ctx, const double* theta0, int32_t n_rb, const int32_t* edges);

/* Relative-binning log-likelihood ratios of n samples (device theta [P][n] -> loglike [n]),
 * with the marginalisations of the context.  The error against mbis_loglike grows with the
 * square of each bin's phase excursion (see mbis_rb_edges).  Errors: MBIS_E_STATE (no
 * set-up), MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_rb_loglike(mbis_ctx* ctx, int64_t n, const double* theta, double* loglike, void* cuda_stream);

/* on != 0: mbis_loglike, and with it the ESS loop (mbis_run_to_ess and the stepwise loop),
 * evaluates the relative-binning likelihood of the context's set-up instead of the exact
 * one, so the importance-sampling loop runs on the faster likelihood (Sec. IV); on = 0
 * restores the exact likelihood.  Proposal refits keep the set-up; mbis_set_metric drops it
 * and turns this off.  A context with this on cannot join a multi-event batch.
 * Errors: MBIS_E_STATE (on without a current set-up), MBIS_E_INVALID. */
mbis_status mbis_rb_use(mbis_ctx* ctx, int32_t on);

/* Coarse bins for relative binning: each bin's largest change of the template's phase
 * relative to the fiducial, over the box theta0 +- n_sigma proposal standard deviations
 * (clipped to the prior), stays below eps_rad, which bounds the chord's error by about
 * eps_rad^2 / 8 of the bin's overlap.  edges (host, max_bins + 1), *n_rb (host).
 * Errors: MBIS_E_STATE, MBIS_E_INVALID (more than max_bins bins). */
mbis_status mbis_rb_edges(const mbis_ctx* ctx, const double* theta0, double n_sigma, double eps_rad, int32_t max_bins,
                          int32_t* edges, int32_t* n_rb);

/* What mbis_set_metric built for the context (diagnostics; not in the paper). */
typedef struct {
  int32_t tables;    /* -1: none yet; 1: one folded table (sky and orientation fixed); 0: per detector */
  int32_t n_rows;    /* rows of the likelihood tables: 1 folded, n_det per detector, 0 none */
  int32_t ff_phase;  /* MBIS_MIXED: 1 when anchor blocks are entered in float-float arithmetic
                        (every phase term below 2^16 turns), 0 in FP64; -1 otherwise */
  int32_t n_blocks;  /* MBIS_MIXED: anchor blocks of the phase plan */
  int32_t P;         /* sampled slots (0 without a metric) */
} mbis_ctx_info;

/* Errors: MBIS_E_INVALID (null argument; reported by mbis_last_error(NULL)). */
mbis_status mbis_get_info(const mbis_ctx* ctx, mbis_ctx_info* out);

/* Running state merged by mbis_reduce(accumulate != 0); mbis_reset_running clears it. */
mbis_status mbis_get_running(const mbis_ctx* ctx, mbis_summary* out);
mbis_status mbis_reset_running(mbis_ctx* ctx);

/* Merge two reducer states (associative; used to combine shards of one event). */
void mbis_merge_summaries(const mbis_summary* a, const mbis_summary* b, mbis_summary* out);

void mbis_destroy(mbis_ctx* ctx);
const char* mbis_last_error(const mbis_ctx* ctx);

/* ---- set-up helpers (not on the per-sample path) ------------------------------------ */

/* Analytic aLIGO-like PSD fit (Ajith 2011) on the grid; out (host, n_bins doubles).
 * The paper names only "Advanced LIGO O3-like" sensitivity (Sec. III A). */
mbis_status mbis_psd_aligo(const mbis_freq_grid* grid, double* out);

/* Synthetic data for one event: d = h(theta_true) (+ noise n_k = sqrt(S_k / (4 df))
 * (g1 + i g2) when add_noise, g from Philox counter (k, det, 1, 0), key = noise_seed).
 * theta_true (host, 11 slots).  strain_out (host, [n_det][n_bins] complex128 interleaved),
 * snr2_out (host, may be NULL): optimal network SNR^2 = sum_det (h|h).  Computed in FP64
 * on the device.  Errors: MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_inject(const mbis_freq_grid* grid, int32_t n_det, const mbis_detector* dets, const double* psd,
                        double gmst_rad, const double* theta_true, uint64_t noise_seed, int32_t add_noise,
                        double* strain_out, double* snr2_out);

/* Fisher matrix Gamma_ij = sum_det (d_i h | d_j h) (the metric of the inner product of
 * Eq. 1, Sec. II A) at theta (host, 11 slots) over slots ids (host, P), by FP64 central
 * differences with absolute steps (host, P), computed on the device.  gamma_out (host,
 * P x P row-major).  Uses the context's PSD, detectors and grid (not its data).
 * Errors: MBIS_E_INVALID, MBIS_E_OOM, MBIS_E_CUDA. */
mbis_status mbis_fisher(mbis_ctx* ctx, const double* theta, int32_t P, const int32_t* ids, const double* steps,
                        double* gamma_out);

/* Settings of the Gaussian proposal in the Fisher metric (mbis_fisher_proposal). */
typedef struct {
  double scale;         /* width scale s: the proposal is N(theta0, s^2 Gamma^-1) (> 0) */
  double box_sigmas;    /* prior box of Mc, q and t_c: theta0 +- box_sigmas s sigma (> 0) */
  double chi_max;       /* prior of chi1z, chi2z: [-chi_max, chi_max] (0 < chi_max < 1 when a spin is sampled) */
  double dmin_mpc, dmax_mpc;  /* prior range of a sampled d_L (0 < dmin < dmax when d_L is sampled) */
} mbis_proposal_options;

/* The Gaussian proposal of Sec. II A from a Fisher matrix: the metric of the inner product
 * of Eq. 1 at the trigger theta0 (host, 11 slots), gamma (host, N x N row-major, N = P +
 * n_marg) over the sampled slots ids (host, P) followed by the slots the likelihood
 * marginalises, marg_ids (host, n_marg; phi_c under phase, d_L under distance
 * marginalisation).  Steps, in this order:
 *   1. the marginalised slots are projected out: G = A - B C^-1 B^T (Schur complement);
 *   2. for slots the data barely constrain (q, spins, angles, a sampled d_L) G gains
 *      12 / width^2 on its diagonal -- the inverse variance of a uniform distribution over
 *      the slot's prior range (q: 2; chi: 2 chi_max; RA, phi_c: 2 pi; dec, psi, iota: pi;
 *      d_L: dmax - dmin) -- so the proposal stays inside the prior;
 *   3. covariance = G^-1 (symmetrised), chol_out = its lower Cholesky factor;
 *   4. mean_out = theta0 on the sampled slots; the prior box lo_out / hi_out is theta0 +-
 *      box_sigmas scale sigma_p for Mc and t_c (and for q, whose lower end is at least 1),
 *      [-chi_max, chi_max] for the spins and the physical range for the other slots.
 * Outputs (host): mean_out [P], chol_out [P x P] row-major lower, lo_out, hi_out [P]: the
 * arguments of mbis_set_metric.  Pure host arithmetic: needs no GPU and no context;
 * failures are reported by mbis_last_error(NULL).
 * Errors: MBIS_E_INVALID (null, repeated or out-of-range slot, bad option, a matrix that
 * is not positive definite). */
mbis_status mbis_proposal_from_fisher(int32_t P, const int32_t* ids, int32_t n_marg, const int32_t* marg_ids,
                                      const double* gamma, const double* theta0, const mbis_proposal_options* opts,
                                      double* mean_out, double* chol_out, double* lo_out, double* hi_out);

/* mbis_fisher at theta0 over ids plus the slots the context marginalises (phi_c with
 * MBIS_MARG_PHASE, d_L with MBIS_MARG_DISTANCE), central-difference steps 1e-6 relative
 * (Mc), 1e-5 relative (d_L), 1e-5 (chi), 1e-7 s (t_c) and 1e-6 otherwise; then
 * mbis_proposal_from_fisher.  Same outputs; a slot may not be both sampled and
 * marginalised.  Errors: as mbis_fisher and mbis_proposal_from_fisher. */
mbis_status mbis_fisher_proposal(mbis_ctx* ctx, const double* theta0, int32_t P, const int32_t* ids,
                                 const mbis_proposal_options* opts, double* mean_out, double* chol_out,
                                 double* lo_out, double* hi_out);

/* Self-test of the bounded device-side wait that every kernel uses on its mbarriers (not
 * in the paper): one thread waits on a barrier that nothing completes, gives up after
 * limit_ns (0 < limit_ns <= 2e9) of GPU wall time and reports *status_out = MBIS_E_TIMEOUT
 * (host), *waited_ns_out (host, nullable) the time it waited.  The context stays usable --
 * this is how a stuck copy or MMA surfaces in the other kernels (as MBIS_E_TIMEOUT from the
 * next mbis_reduce) instead of a hang.  Returns MBIS_E_INVALID or MBIS_E_CUDA on failure. */
mbis_status mbis_debug_wait_timeout(uint64_t limit_ns, int32_t* status_out, uint64_t* waited_ns_out);

/* Self-test of the float-float sine and cosine that the time-marginalised kernel's
 * per-sample set-up uses for the sky and orientation angles (not in the paper): for n
 * angles x (device, FP64) writes sin x and cos x (device, FP64, nullable each) as that
 * kernel computes them (a Cody-Waite reduction by pi/2 and the Taylor series in float-float
 * arithmetic: absolute error below ~1e-13 for |x| < 8 pi, growing as |x| 1e-16 beyond it,
 * from the FP64 pi/2 of the reduction; angles with |x| >= 2^20 take the library's FP64
 * sincos).  Errors: MBIS_E_INVALID (n < 0, null x with n > 0), MBIS_E_CUDA. */
mbis_status mbis_debug_ff_sincos(int64_t n, const double* x, double* sin_out, double* cos_out, void* cuda_stream);

/* Self-test of the time-marginalised kernel's float-float per-sample set-up (not in the
 * paper): for n parameter sets params (device, [7][n]: Mc, q, chi1, chi2, t_c, phi_c, d_L)
 * on the grid (f_lo, df, n_bins), out (device, [2][12][n]) receives the FP64 set-up of the
 * mixed kernels (block 0) and the float-float one (block 1): the phase coefficients C_0..C_8
 * (turns), the constant, the amplitude at d_L and the ISCO cut (as a double).
 * Errors: MBIS_E_INVALID, MBIS_E_CUDA. */
mbis_status mbis_debug_setup_pair(int64_t n, const double* params, double f_lo, double df, int32_t n_bins,
                                  double* out, void* cuda_stream);

/* Library build/version string. */
const char* mbis_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MBIS_H */
