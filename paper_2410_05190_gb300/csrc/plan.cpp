// plan.cpp -- host-side anchor-block plan of the mixed-precision phase.
//
// The TaylorF2 phase reaches ~10^4 turns at 20 Hz for a neutron-star binary, far beyond
// what FP32 resolves, while the GB300 executes FP64 at a small fraction of its FP32 rate.
// The bins are therefore cut into blocks.  In block [k0, k1) with centre bin kc the phase is
//   Psi_k/2pi = X + (k - kc) Y + sum_j C_j R_j(k - kc),
// where X and Y (value and per-bin slope at kc) are taken in FP64 once per block and sample
// and reduced modulo one turn, and R_j, the remainder of basis function j beyond its tangent
// at f_kc, is a small smooth function that a degree-5 polynomial in w = k - kc represents
// to well below 1e-7 turns.  Blocks grow as long as (i) sum_j max|C_j| * fit_error_j stays
// under tol and (ii) sum_j max|C_j| * max|R_j| stays under rmax, so that the FP32 remainder
// keeps ~1e-7-turn resolution.  max|C_j| is bounded over the prior box by the caller.
#include <algorithm>
#include <cmath>
#include <list>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace mbis {
namespace {

// LU factorisation with partial pivoting of the (n x n) matrix A in place (whole rows swapped,
// piv: the swap of each step), then solves for any number of right-hand sides
void lu_factor(int n, double* A, int* piv) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    piv[c] = p;
    if (p != c)
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / A[c * n + c];
      A[r * n + c] = f;
      for (int k = c + 1; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
    }
  }
}

void lu_solve(int n, const double* LU, const int* piv, double* b) {
  for (int c = 0; c < n; ++c)
    if (piv[c] != c) std::swap(b[c], b[piv[c]]);
  for (int c = 0; c < n; ++c)
    for (int r = c + 1; r < n; ++r) b[r] -= LU[r * n + c] * b[c];
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= LU[c * n + k] * b[k];
    b[c] = s / LU[c * n + c];
  }
}

struct Fit {
  AnchorBlock blk;
  double err_bound, r_bound;
};

// The basis functions with a remainder (B_8 = f is linear)
constexpr int kRemBasis = kNumBasis - 1;

// The fit of one block; its error is checked on every bin, or on max_pts evenly spaced bins.
Fit fit_block(const PlanInput& in, int32_t k0, int32_t S, int32_t max_pts) {
  const int D = in.deg + 1;
  constexpr int DM = kRemDegMax + 1;
  Fit out = {};
  AnchorBlock& b = out.blk;
  b.k0 = k0;
  b.k1 = k0 + S;
  b.kc = k0 + (S - 1) / 2;
  b.pad = 0;
  const double fc = in.f_lo + (double)b.kc * in.df;
  basis_all(fc, b.B);
  for (int j = 0; j < kNumBasis; ++j) {
    b.dB[j] = basis_deriv(j, fc) * in.df;
    const float bh = (float)b.B[j], dbh = (float)b.dB[j];
    b.Bq[j] = make_float4(bh, (float)(b.B[j] - (double)bh), dbh, (float)(b.dB[j] - (double)dbh));
  }
  // remainders of every basis function beyond its tangent at fc, at offset w
  auto rem_all = [&](double w, double* r) {
    double v[kNumBasis];
    basis_all(fc + w * in.df, v);
    for (int j = 0; j < kRemBasis; ++j) r[j] = v[j] - b.B[j] - w * b.dB[j];
  };
  const double wa = (double)(k0 - b.kc), wb = (double)(k0 + S - 1 - b.kc);
  const double h = std::max(1.0, std::max(std::fabs(wa), std::fabs(wb)));
  const double mid = 0.5 * (wa + wb), half = std::max(0.5 * (wb - wa), 0.5);
  // interpolate at Chebyshev points of the block, monomials in u = w / h: one Vandermonde
  // factorisation serves every basis function
  double V[DM * DM], y[kRemBasis][DM];
  int piv[DM];
  for (int i = 0; i < D; ++i) {
    const double w = mid + half * std::cos(kPi * (i + 0.5) / D);
    const double u = w / h;
    double p = 1.0;
    for (int m = 0; m < D; ++m) {
      V[i * D + m] = p;
      p *= u;
    }
    double r[kRemBasis];
    rem_all(w, r);
    for (int j = 0; j < kRemBasis; ++j) y[j][i] = r[j];
  }
  lu_factor(D, V, piv);
  for (int j = 0; j < kRemBasis; ++j) {
    lu_solve(D, V, piv, y[j]);
    double hm = 1.0;
    for (int m = 0; m < D; ++m) {
      b.E[j][m] = (float)(y[j][m] / hm);
      hm *= h;
    }
  }
  // error of the FP32-stored polynomials on the block's bins (all, or max_pts evenly spaced)
  double emax[kRemBasis] = {}, rmax[kRemBasis] = {};
  const int32_t npts = std::min<int32_t>(S, max_pts);
  for (int32_t i = 0; i < npts; ++i) {
    const int32_t kk = (npts == S) ? k0 + i : k0 + (int32_t)std::llround((double)i * (S - 1) / (npts - 1));
    const double w = (double)(kk - b.kc);
    double r[kRemBasis];
    rem_all(w, r);
    for (int j = 0; j < kRemBasis; ++j) {
      double p = 0.0;
      for (int m = D - 1; m >= 0; --m) p = p * w + (double)b.E[j][m];
      emax[j] = std::max(emax[j], std::fabs(p - r[j]));
      rmax[j] = std::max(rmax[j], std::fabs(r[j]));
    }
  }
  out.err_bound = 0.0;
  out.r_bound = 0.0;
  for (int j = 0; j < kRemBasis; ++j) {
    out.err_bound += in.cmax[j] * emax[j];
    out.r_bound += in.cmax[j] * rmax[j];
  }
  return out;
}

constexpr int32_t kSearchPoints = 33, kCheckPoints = 257;

std::vector<AnchorBlock> build_plan(const PlanInput& in) {
  std::vector<AnchorBlock> blocks;
  int32_t k0 = 0;
  int32_t guess = 64;
  while (k0 < in.n_bins) {
    const int32_t remaining = in.n_bins - k0;
    const int32_t cap = std::min(remaining, in.max_block);
    // the search checks 33 bins per trial block; the chosen size is then verified on 257
    // (every bin of a shorter block) and shrunk until that holds
    auto ok_at = [&](int32_t S, int32_t pts) {
      const Fit f = fit_block(in, k0, S, pts);
      return f.err_bound <= in.tol_turns && f.r_bound <= in.rmax_turns;
    };
    auto ok = [&](int32_t S) { return ok_at(S, kSearchPoints); };
    int32_t good = std::min<int32_t>(cap, 8);  // short blocks are interpolated exactly
    if (good < remaining && (good & 1)) good -= 1;
    int32_t S = std::min(cap, std::max(good, guess));
    int32_t bad = -1;
    if (ok(S)) {
      good = S;
      while (good < cap) {
        S = std::min(cap, good * 2);
        if (ok(S)) {
          good = S;
        } else {
          bad = S;
          break;
        }
      }
    } else {
      bad = S;
    }
    if (bad > 0) {
      while (bad - good > 1) {
        const int32_t m = good + (bad - good) / 2;
        if (ok(m)) good = m; else bad = m;
      }
    }
    while (good > 8 && !ok_at(good, kCheckPoints)) good -= std::max<int32_t>(2, good / 16);
    // even sizes keep every block start even, so the kernel can take bins in pairs
    if (good < remaining && good > 2) good &= ~1;
    blocks.push_back(fit_block(in, k0, good, kCheckPoints).blk);
    k0 += good;
    guess = good;
  }
  return blocks;
}

bool same_input(const PlanInput& a, const PlanInput& b) {
  if (a.f_lo != b.f_lo || a.df != b.df || a.n_bins != b.n_bins || a.tol_turns != b.tol_turns ||
      a.rmax_turns != b.rmax_turns || a.max_block != b.max_block || a.deg != b.deg)
    return false;
  for (int j = 0; j < kNumBasis; ++j)
    if (a.cmax[j] != b.cmax[j]) return false;
  return true;
}

// Plans of the most recent inputs, shared by every context of the process: a plan depends
// only on the grid, the coefficient bounds of the prior box and the tolerances, which the
// contexts of one analysis (events on one grid, the served stream's requests) repeat.
constexpr size_t kPlanCacheSize = 8;
std::mutex g_plan_mutex;
std::list<std::pair<PlanInput, std::vector<AnchorBlock>>> g_plans;  // most recent first

}  // namespace

std::vector<AnchorBlock> plan_anchor_blocks(const PlanInput& in) {
  {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it)
      if (same_input(it->first, in)) {
        g_plans.splice(g_plans.begin(), g_plans, it);
        return g_plans.front().second;
      }
  }
  std::vector<AnchorBlock> plan = build_plan(in);
  std::lock_guard<std::mutex> lock(g_plan_mutex);
  g_plans.emplace_front(in, plan);
  if (g_plans.size() > kPlanCacheSize) g_plans.pop_back();
  return plan;
}

}  // namespace mbis
