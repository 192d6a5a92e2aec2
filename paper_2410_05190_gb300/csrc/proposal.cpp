// proposal.cpp -- the Gaussian proposal in the Fisher metric at a trigger (Sec. II A):
// the metric of the inner product of Eq. 1 at the trigger, the marginalised slots projected
// out, a weak prior-width term for directions the data barely constrain, and the prior box.
// Host arithmetic on a P x P matrix (P <= 11): not on the per-sample path.
#include <cmath>
#include <cstring>
#include <string>

#include "internal.h"

using namespace mbis;

namespace {

constexpr double kTwoPiD = 6.283185307179586476925286766559;
constexpr double kPiD = 3.1415926535897932384626433832795;
constexpr int kMaxDim = kNumSlots;

// In-place Cholesky factor of the n x n symmetric positive-definite matrix a (row-major,
// leading dimension ld): the lower triangle becomes L with a = L L^T, the strict upper
// triangle is zeroed.  False when a pivot is not positive (the matrix is not positive
// definite to working precision).
bool cholesky(double* a, int n, int ld) {
  for (int j = 0; j < n; ++j) {
    double d = a[j * ld + j];
    for (int k = 0; k < j; ++k) d -= a[j * ld + k] * a[j * ld + k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d);
    a[j * ld + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * ld + j];
      for (int k = 0; k < j; ++k) s -= a[i * ld + k] * a[j * ld + k];
      a[i * ld + j] = s / ljj;
    }
    for (int i = 0; i < j; ++i) a[i * ld + j] = 0.0;
  }
  return true;
}

// x = A^-1 b for A = L L^T (L from cholesky), one right-hand side of length n.
void chol_solve(const double* L, int n, int ld, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * ld + k] * x[k];
    x[i] = s / L[i * ld + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * ld + i] * x[k];
    x[i] = s / L[i * ld + i];
  }
}

// Variance of a uniform distribution over the slot's prior range, as the width^2/12 of the
// regularising term; 0 for slots the data always constrain (Mc, t_c).
double prior_width(int id, const mbis_proposal_options& o) {
  switch (id) {
    case kQ: return 2.0;
    case kChi1:
    case kChi2: return 2.0 * o.chi_max;
    case kRa:
    case kPhic: return kTwoPiD;
    case kDec:
    case kPsi:
    case kIota: return kPiD;
    case kDl: return o.dmax_mpc - o.dmin_mpc;
    default: return 0.0;
  }
}

mbis_status bad(const std::string& msg) {
  set_last_error(msg);
  return MBIS_E_INVALID;
}

}  // namespace

extern "C" {

mbis_status mbis_proposal_from_fisher(int32_t P, const int32_t* ids, int32_t n_marg, const int32_t* marg_ids,
                                      const double* gamma, const double* theta0, const mbis_proposal_options* o,
                                      double* mean_out, double* chol_out, double* lo_out, double* hi_out) {
  const char* fn = "mbis_proposal_from_fisher: ";
  if (!ids || !gamma || !theta0 || !o || !mean_out || !chol_out || !lo_out || !hi_out || (n_marg > 0 && !marg_ids))
    return bad(std::string(fn) + "null argument");
  if (P < 1 || n_marg < 0 || P + n_marg > kMaxDim) return bad(std::string(fn) + "need 1 <= P and P + n_marg <= 11");
  if (!(o->scale > 0.0) || !(o->box_sigmas > 0.0)) return bad(std::string(fn) + "need scale > 0, box_sigmas > 0");
  bool seen[kNumSlots] = {};
  const int N = P + n_marg;
  for (int i = 0; i < N; ++i) {
    const int id = i < P ? ids[i] : marg_ids[i - P];
    if (id < 0 || id >= kNumSlots || seen[id]) return bad(std::string(fn) + "slot ids must be distinct and < 11");
    seen[id] = true;
  }
  // the spin and distance bounds matter only where those slots are sampled
  bool spin = false, dist = false;
  for (int p = 0; p < P; ++p) {
    spin = spin || ids[p] == kChi1 || ids[p] == kChi2;
    dist = dist || ids[p] == kDl;
  }
  if (spin && !(o->chi_max > 0.0 && o->chi_max < 1.0))
    return bad(std::string(fn) + "a sampled spin needs 0 < chi_max < 1");
  if (dist && !(o->dmin_mpc > 0.0 && o->dmax_mpc > o->dmin_mpc))
    return bad(std::string(fn) + "a sampled distance needs 0 < dmin < dmax");
  for (int i = 0; i < N * N; ++i)
    if (!std::isfinite(gamma[i])) return bad(std::string(fn) + "non-finite Fisher matrix entry");

  // Schur complement of the marginalised block: G = A - B C^-1 B^T
  double G[kMaxDim * kMaxDim];
  for (int r = 0; r < P; ++r)
    for (int s = 0; s < P; ++s) G[r * P + s] = gamma[r * N + s];
  if (n_marg > 0) {
    double C[kMaxDim * kMaxDim];
    for (int r = 0; r < n_marg; ++r)
      for (int s = 0; s < n_marg; ++s) C[r * n_marg + s] = gamma[(P + r) * N + P + s];
    if (!cholesky(C, n_marg, n_marg))
      return bad(std::string(fn) + "the marginalised slots' block of the Fisher matrix is not positive definite");
    for (int s = 0; s < P; ++s) {
      double x[kMaxDim];  // C^-1 B^T[:, s]
      for (int r = 0; r < n_marg; ++r) x[r] = gamma[s * N + P + r];
      chol_solve(C, n_marg, n_marg, x);
      for (int r = 0; r < P; ++r) {
        double bx = 0.0;
        for (int k = 0; k < n_marg; ++k) bx += gamma[r * N + P + k] * x[k];
        G[r * P + s] -= bx;
      }
    }
  }
  // weak Gaussian term of the prior's width: variance width^2 / 12 per poorly measured slot
  for (int p = 0; p < P; ++p) {
    const double w = prior_width(ids[p], *o);
    if (w > 0.0) G[p * P + p] += 12.0 / (w * w);
  }
  // covariance = G^-1 (symmetrised), then its Cholesky factor
  double Lg[kMaxDim * kMaxDim];
  for (int r = 0; r < P; ++r)
    for (int s = 0; s < P; ++s) Lg[r * P + s] = 0.5 * (G[r * P + s] + G[s * P + r]);
  if (!cholesky(Lg, P, P)) return bad(std::string(fn) + "the projected Fisher matrix is not positive definite");
  double cov[kMaxDim * kMaxDim];
  for (int s = 0; s < P; ++s) {
    double x[kMaxDim] = {};
    x[s] = 1.0;
    chol_solve(Lg, P, P, x);
    for (int r = 0; r < P; ++r) cov[r * P + s] = x[r];
  }
  for (int r = 0; r < P; ++r)
    for (int s = 0; s < r; ++s) cov[r * P + s] = cov[s * P + r] = 0.5 * (cov[r * P + s] + cov[s * P + r]);
  double L[kMaxDim * kMaxDim];
  std::memcpy(L, cov, sizeof(double) * P * P);
  if (!cholesky(L, P, P)) return bad(std::string(fn) + "the proposal covariance is not positive definite");

  // mean at the trigger; prior box: +-box_sigmas proposal sigmas for Mc, q, t_c (q >= 1),
  // the physical range for the others
  for (int p = 0; p < P; ++p) {
    const int id = ids[p];
    const double x0 = theta0[id];
    const double sig = std::sqrt(cov[p * P + p]) * o->scale;
    double lo = 0.0, hi = 0.0;
    switch (id) {
      case kChi1:
      case kChi2: lo = -o->chi_max; hi = o->chi_max; break;
      case kQ: lo = std::fmax(1.0, x0 - o->box_sigmas * sig); hi = x0 + o->box_sigmas * sig; break;
      case kMc:
      case kTc: lo = x0 - o->box_sigmas * sig; hi = x0 + o->box_sigmas * sig; break;
      case kRa:
      case kPhic: lo = 0.0; hi = kTwoPiD; break;
      case kPsi: lo = 0.0; hi = kPiD; break;
      case kDec: lo = -0.5 * kPiD; hi = 0.5 * kPiD; break;
      case kIota: lo = 0.0; hi = kPiD; break;
      case kDl: lo = o->dmin_mpc; hi = o->dmax_mpc; break;
    }
    mean_out[p] = x0;
    lo_out[p] = lo;
    hi_out[p] = hi;
  }
  std::memcpy(chol_out, L, sizeof(double) * P * P);
  return MBIS_OK;
}

mbis_status mbis_fisher_proposal(mbis_ctx* c, const double* theta0, int32_t P, const int32_t* ids,
                                 const mbis_proposal_options* o, double* mean_out, double* chol_out, double* lo_out,
                                 double* hi_out) {
  if (!c) return bad("mbis_fisher_proposal: null context");
  if (!theta0 || !ids || !o || P < 1 || P > kNumSlots) {
    c->err = "mbis_fisher_proposal: bad argument";
    return bad(c->err);
  }
  // slots the likelihood marginalises are projected out of the metric
  int32_t all[kNumSlots];
  int N = 0;
  for (int p = 0; p < P; ++p) all[N++] = ids[p];
  const uint32_t marg = c->opts.marg;
  if (marg & MBIS_MARG_PHASE) all[N++] = kPhic;
  if (marg & MBIS_MARG_DISTANCE) all[N++] = kDl;
  if (N > kNumSlots) {
    c->err = "mbis_fisher_proposal: a marginalised slot is also sampled";
    return bad(c->err);
  }
  // central-difference steps: relative for Mc and d_L, absolute otherwise
  double steps[kNumSlots];
  for (int i = 0; i < N; ++i) {
    const int id = all[i];
    if (id < 0 || id >= kNumSlots) {
      c->err = "mbis_fisher_proposal: bad slot id";
      return bad(c->err);
    }
    double h = 1e-6;
    if (id == kChi1 || id == kChi2 || id == kDl) h = 1e-5;
    if (id == kTc) h = 1e-7;
    steps[i] = (id == kMc || id == kDl) ? h * theta0[id] : h;
  }
  double gamma[kNumSlots * kNumSlots];
  mbis_status st = mbis_fisher(c, theta0, N, all, steps, gamma);
  if (st != MBIS_OK) return st;
  st = mbis_proposal_from_fisher(P, ids, N - P, all + P, gamma, theta0, o, mean_out, chol_out, lo_out, hi_out);
  if (st != MBIS_OK) c->err = mbis_last_error(nullptr);
  return st;
}

}  // extern "C"
