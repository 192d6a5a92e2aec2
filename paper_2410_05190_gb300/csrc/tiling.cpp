// tiling.cpp -- the tiled proposal's host object (template bank, prior-volume tiles,
// mixture) and its C ABI (Sec. II; App. A).  All per-point arithmetic runs in the
// kernels of k_tiling.cu; the host takes the template-placement decisions in candidate
// order from FP64 matches computed on the device, and manages memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tiling.h"

using mbis::TilingGrid;
using mbis::TilingSpace;

struct mbis_tiling {
  TilingSpace sp = {};
  double f_lo = 0.0, df = 0.0;
  int32_t n_bins = 0, K = 0, n_kb = 0;
  double wref = 1.0;
  double* d_w = nullptr;      // [K]
  double* d_w2sum = nullptr;  // [K + 1]
  float* d_bins = nullptr;    // [n_kb * 8][kBinRecord]
  int32_t* d_err = nullptr;
  // bank
  int32_t T = 0, cap = 0;
  std::vector<double> tx, tq;
  std::vector<int32_t> cand_idx;
  double2* d_rows = nullptr;  // [cap][K]
  double2* d_kmaj = nullptr;  // [K][cap]
  void* d_tiles = nullptr;    // FP16 [n_pass][n_kb][2][256 x 64]
  int32_t n_pass = 0;
  int32_t* d_perm = nullptr;  // [n_pass * 256] templates by pass slot (ordered by live-bin count), -1 pads
  std::vector<int32_t> nkb_pass;
  // scratch of the assignment's sample ordering (grown on demand)
  int64_t scr_n = 0;
  float4* d_rec = nullptr;
  int32_t *d_kc = nullptr, *d_order = nullptr, *d_shist = nullptr, *d_scount = nullptr, *d_soffset = nullptr,
          *d_snbad = nullptr;
  // pool
  int64_t N = 0;
  double* d_pool = nullptr;   // [2][N]
  int32_t *d_tile_of = nullptr, *d_members = nullptr, *d_hist = nullptr, *d_count = nullptr, *d_offset = nullptr,
          *d_nbad = nullptr;
  std::vector<int64_t> counts;
  // mixture
  bool has_mix = false;
  double *d_c = nullptr, *d_mix = nullptr, *d_ll = nullptr;
  int32_t* d_flag = nullptr;
  std::string err;

  TilingGrid grid() const {
    TilingGrid g;
    g.f_lo = f_lo;
    g.df = df;
    g.K = K;
    g.n_kb = n_kb;
    g.w = d_w;
    g.w2sum = d_w2sum;
    g.wref = wref;
    g.inv_wref2 = 1.0 / (wref * wref);
    return g;
  }
};

namespace {

constexpr int32_t kBankBatch = 1024;

mbis_status tfail(mbis_tiling* t, mbis_status st, const std::string& msg) {
  if (t)
    t->err = msg;
  else
    mbis::set_last_error(msg);
  return st;
}

#define T_TRY(t, expr)                                                                          \
  do {                                                                                          \
    const cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                      \
      return tfail((t), e_ == cudaErrorMemoryAllocation ? MBIS_E_OOM : MBIS_E_CUDA,             \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

template <typename P>
void tfree(P*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void drop_mixture(mbis_tiling* t) {
  tfree(t->d_c);
  tfree(t->d_mix);
  tfree(t->d_ll);
  tfree(t->d_flag);
  t->has_mix = false;
}

void drop_pool(mbis_tiling* t) {
  drop_mixture(t);
  tfree(t->d_pool);
  tfree(t->d_tile_of);
  tfree(t->d_members);
  tfree(t->d_hist);
  tfree(t->d_count);
  tfree(t->d_offset);
  tfree(t->d_nbad);
  t->N = 0;
  t->counts.clear();
}

void drop_bank(mbis_tiling* t) {
  drop_pool(t);
  tfree(t->d_rows);
  tfree(t->d_kmaj);
  tfree(t->d_tiles);
  tfree(t->d_perm);
  t->nkb_pass.clear();
  t->T = t->cap = t->n_pass = 0;
  t->tx.clear();
  t->tq.clear();
  t->cand_idx.clear();
}

void drop_scratch(mbis_tiling* t) {
  tfree(t->d_kc);
  tfree(t->d_rec);
  tfree(t->d_order);
  tfree(t->d_shist);
  tfree(t->d_scount);
  tfree(t->d_soffset);
  tfree(t->d_snbad);
  t->scr_n = 0;
}

bool in_space(const TilingSpace& s, double x, double q) {
  return x >= s.x_lo && x < s.x_hi && q >= s.q_lo && q <= s.q_hi;
}

void physical(const TilingSpace& sp, double x, double q, double* mc, double* qp) {
  if (sp.mc_period > 0.0) {
    double r = std::fmod(x, sp.mc_period);
    if (r < 0.0) r += sp.mc_period;
    *mc = sp.mc_base + r;
  } else {
    *mc = x;
  }
  *qp = q >= 1.0 ? q : 1.0 / q;
}

// grow the bank's FP64 storage to hold `need` templates
mbis_status grow(mbis_tiling* t, int32_t need, int32_t max_t) {
  if (need <= t->cap) return MBIS_OK;
  const int32_t nc = std::max(need, std::min(max_t, std::max(2 * t->cap, 256)));
  double2 *rows = nullptr, *kmaj = nullptr;
  if (cudaMalloc(&rows, sizeof(double2) * (size_t)nc * t->K) != cudaSuccess ||
      cudaMalloc(&kmaj, sizeof(double2) * (size_t)nc * t->K) != cudaSuccess) {
    tfree(rows);
    tfree(kmaj);
    return tfail(t, MBIS_E_OOM, "mbis_tiling_bank: out of device memory");
  }
  if (t->T > 0) {
    cudaError_t e = cudaMemcpy(rows, t->d_rows, sizeof(double2) * (size_t)t->T * t->K, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy2D(kmaj, sizeof(double2) * nc, t->d_kmaj, sizeof(double2) * t->cap, sizeof(double2) * t->T, t->K,
                       cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      tfree(rows);
      tfree(kmaj);
      return tfail(t, MBIS_E_CUDA, std::string("mbis_tiling_bank: ") + cudaGetErrorString(e));
    }
  }
  tfree(t->d_rows);
  tfree(t->d_kmaj);
  t->d_rows = rows;
  t->d_kmaj = kmaj;
  t->cap = nc;
  return MBIS_OK;
}

}  // namespace

extern "C" {

mbis_status mbis_tiling_create(const mbis_freq_grid* grid, const double* psd, const mbis_tiling_space* space,
                               mbis_tiling** out) {
  if (!out) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: null out");
  *out = nullptr;
  if (!grid || !psd || !space) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: null argument");
  if (!(grid->n_bins >= 1 && grid->df > 0.0 && grid->f_lo > 0.0 && std::isfinite(grid->df) &&
        std::isfinite(grid->f_lo)))
    return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: need n_bins >= 1, df > 0, f_lo > 0");
  const mbis_tiling_space& s = *space;
  if (!(s.x_lo < s.x_hi) || !std::isfinite(s.x_lo) || !std::isfinite(s.x_hi) || !(s.q_lo > 0.0) ||
      !(s.q_lo <= s.q_hi) || !std::isfinite(s.q_hi) || !(s.mc_period >= 0.0) || !std::isfinite(s.mc_period) ||
      !(std::fabs(s.chi1) < 1.0) || !(std::fabs(s.chi2) < 1.0))
    return tfail(nullptr, MBIS_E_INVALID,
                 "mbis_tiling_create: bad space (need x_lo < x_hi, 0 < q_lo <= q_hi, mc_period >= 0, |chi| < 1)");
  double mc_lo, mc_hi;
  if (s.mc_period > 0.0) {
    if (!(s.mc_base > 0.0)) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: need mc_base > 0");
    mc_lo = s.mc_base;
    mc_hi = s.mc_base + s.mc_period;
  } else {
    if (!(s.x_lo > 0.0)) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: need x_lo > 0 (chirp mass)");
    mc_lo = s.x_lo;
    mc_hi = s.x_hi;
  }
  const double q_min = (s.q_lo <= 1.0 && s.q_hi >= 1.0) ? 1.0 : (s.q_lo > 1.0 ? s.q_lo : 1.0 / s.q_hi);
  const double q_max = std::max(s.q_hi, 1.0 / s.q_lo);
  // the total mass grows with Mc and with q >= 1: the lightest point reaches the most bins
  const int32_t K = mbis::live_bins_m(mbis::total_mass_seconds(mc_lo, q_min), grid->f_lo, grid->df, grid->n_bins);
  const int32_t K_heavy =
      mbis::live_bins_m(mbis::total_mass_seconds(mc_hi, q_max), grid->f_lo, grid->df, grid->n_bins);
  if (K < 1 || K_heavy < 1)
    return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: part of the space has no bin below its ISCO");
  std::vector<double> w(K), w2(K);
  double wref = 0.0;
  for (int32_t k = 0; k < K; ++k) {
    if (!(psd[k] > 0.0) || !std::isfinite(psd[k]))
      return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_create: PSD must be > 0 on the bins the space reaches");
    const double f = grid->f_lo + (double)k * grid->df;
    w[k] = std::pow(f, -7.0 / 6.0) / std::sqrt(psd[k]);
    w2[k] = w[k] * w[k];
    wref = std::max(wref, w[k]);
  }
  mbis_tiling* t = new mbis_tiling();
  t->sp = {s.x_lo, s.x_hi, s.mc_period, s.mc_base, s.q_lo, s.q_hi, s.chi1, s.chi2};
  t->f_lo = grid->f_lo;
  t->df = grid->df;
  t->n_bins = grid->n_bins;
  t->K = K;
  t->n_kb = (K + mbis::kTileBins - 1) / mbis::kTileBins;
  t->wref = wref;
  double* d_w2 = nullptr;
  auto fail_free = [&](mbis_status st, const std::string& msg) {
    tfree(d_w2);
    mbis_tiling_destroy(t);
    return tfail(nullptr, st, msg);
  };
  if (cudaMalloc(&t->d_w, sizeof(double) * K) != cudaSuccess ||
      cudaMalloc(&t->d_w2sum, sizeof(double) * (K + 1)) != cudaSuccess ||
      cudaMalloc(&d_w2, sizeof(double) * K) != cudaSuccess ||
      cudaMalloc(&t->d_bins, sizeof(float) * (size_t)t->n_kb * (mbis::kTileBins / 2) * mbis::kBinRecord) != cudaSuccess ||
      cudaMalloc(&t->d_err, sizeof(int32_t)) != cudaSuccess)
    return fail_free(MBIS_E_OOM, "mbis_tiling_create: out of device memory");
  cudaError_t e = cudaMemcpy(t->d_w, w.data(), sizeof(double) * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_w2, w2.data(), sizeof(double) * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->d_err, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = mbis::launch_prefix_rows(d_w2, 1, K, t->d_w2sum, nullptr);
  if (e == cudaSuccess) e = mbis::launch_tiling_bin_records(t->grid(), 1.0 / wref, t->d_bins, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail_free(MBIS_E_CUDA, std::string("mbis_tiling_create: ") + cudaGetErrorString(e));
  tfree(d_w2);
  *out = t;
  return MBIS_OK;
}

void mbis_tiling_destroy(mbis_tiling* t) {
  if (!t) return;
  drop_bank(t);
  drop_scratch(t);
  tfree(t->d_w);
  tfree(t->d_w2sum);
  tfree(t->d_bins);
  tfree(t->d_err);
  delete t;
}

const char* mbis_tiling_last_error(const mbis_tiling* t) { return t ? t->err.c_str() : mbis_last_error(nullptr); }

mbis_status mbis_tiling_bank(mbis_tiling* t, int64_t n_cand, const double* cand, double min_match, int64_t stop_after,
                             int32_t max_templates, int32_t* n_templates, int64_t* n_used) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_bank: null tiling");
  if (n_cand < 1 || !cand) return tfail(t, MBIS_E_INVALID, "mbis_tiling_bank: need n_cand >= 1 candidates");
  if (!(min_match > 0.0 && min_match < 1.0)) return tfail(t, MBIS_E_INVALID, "mbis_tiling_bank: need 0 < min_match < 1");
  if (stop_after < 1) return tfail(t, MBIS_E_INVALID, "mbis_tiling_bank: need stop_after >= 1");
  if (max_templates < 1 || max_templates > mbis::kTilingMaxTemplates)
    return tfail(t, MBIS_E_INVALID, "mbis_tiling_bank: max_templates must be 1..16384");
  for (int64_t i = 0; i < n_cand; ++i)
    if (!in_space(t->sp, cand[i], cand[n_cand + i]))
      return tfail(t, MBIS_E_INVALID, "mbis_tiling_bank: candidate " + std::to_string(i) + " is outside the space");
  drop_bank(t);
  const int32_t K = t->K;
  const TilingGrid g = t->grid();
  double* d_cpts = nullptr;
  double2 *d_crow = nullptr, *d_ckm = nullptr;
  double *d_out1 = nullptr, *d_out2 = nullptr;
  int32_t* d_idx = nullptr;
  auto cleanup = [&]() {
    tfree(d_cpts);
    tfree(d_crow);
    tfree(d_ckm);
    tfree(d_out1);
    tfree(d_out2);
    tfree(d_idx);
  };
  {
    const int32_t B = kBankBatch;
    if (cudaMalloc(&d_cpts, sizeof(double) * 2 * B) != cudaSuccess ||
        cudaMalloc(&d_crow, sizeof(double2) * (size_t)B * K) != cudaSuccess ||
        cudaMalloc(&d_ckm, sizeof(double2) * (size_t)B * K) != cudaSuccess ||
        cudaMalloc(&d_out1, sizeof(double) * (size_t)B * max_templates) != cudaSuccess ||
        cudaMalloc(&d_out2, sizeof(double) * (size_t)B * B) != cudaSuccess ||
        cudaMalloc(&d_idx, sizeof(int32_t) * B) != cudaSuccess) {
      cleanup();
      return tfail(t, MBIS_E_OOM, "mbis_tiling_bank: out of device memory");
    }
  }
  mbis_status st = MBIS_OK;
  std::vector<double> hp(2 * kBankBatch), h1, h2((size_t)kBankBatch * kBankBatch);
  std::vector<int32_t> acc;
  int64_t i = 0, run = 0;
  while (i < n_cand && t->T < max_templates && run < stop_after) {
    const int32_t B = (int32_t)std::min<int64_t>(kBankBatch, n_cand - i);
    for (int32_t c = 0; c < B; ++c) {
      hp[c] = cand[i + c];
      hp[B + c] = cand[n_cand + i + c];
    }
    cudaError_t e = cudaMemcpy(d_cpts, hp.data(), sizeof(double) * 2 * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mbis::launch_tiling_waveforms(t->sp, g, B, d_cpts, d_crow, d_ckm, B, 0, nullptr);
    const int32_t T = t->T;
    if (e == cudaSuccess && T > 0) e = mbis::launch_tiling_absdots(B, d_crow, T, t->d_kmaj, t->cap, K, d_out1, nullptr);
    if (e == cudaSuccess) e = mbis::launch_tiling_absdots(B, d_crow, B, d_ckm, B, K, d_out2, nullptr);
    if (e == cudaSuccess && T > 0) {
      h1.resize((size_t)B * T);
      e = cudaMemcpy(h1.data(), d_out1, sizeof(double) * (size_t)B * T, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h2.data(), d_out2, sizeof(double) * (size_t)B * B, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      st = tfail(t, MBIS_E_CUDA, std::string("mbis_tiling_bank: ") + cudaGetErrorString(e));
      break;
    }
    // placement decisions in candidate order
    acc.clear();
    int32_t c = 0;
    for (; c < B; ++c) {
      if (run >= stop_after || T + (int32_t)acc.size() >= max_templates) break;
      double best = 0.0;
      for (int32_t j = 0; j < T; ++j) best = std::max(best, h1[(size_t)c * T + j]);
      for (int32_t a : acc) best = std::max(best, h2[(size_t)c * B + a]);
      if (T + (int32_t)acc.size() == 0 || best < min_match) {
        acc.push_back(c);
        run = 0;
      } else {
        ++run;
      }
    }
    if (!acc.empty()) {
      st = grow(t, T + (int32_t)acc.size(), max_templates);
      if (st != MBIS_OK) break;
      e = cudaMemcpy(d_idx, acc.data(), sizeof(int32_t) * acc.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = mbis::launch_tiling_append((int32_t)acc.size(), d_idx, d_crow, K, t->d_rows, T, t->d_kmaj, t->cap,
                                       nullptr);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) {
        st = tfail(t, MBIS_E_CUDA, std::string("mbis_tiling_bank: ") + cudaGetErrorString(e));
        break;
      }
      for (int32_t a : acc) {
        t->tx.push_back(cand[i + a]);
        t->tq.push_back(cand[n_cand + i + a]);
        t->cand_idx.push_back((int32_t)(i + a));
      }
      t->T = T + (int32_t)acc.size();
    }
    i += c;
  }
  cleanup();
  if (st != MBIS_OK) {
    drop_bank(t);
    return st;
  }
  // TF32 template tiles of the tensor-core assignment: templates ordered by live-bin count
  // (most first) into passes of 256, each pass running over the K-blocks its templates reach
  {
    const int32_t T = t->T;
    std::vector<int32_t> kc(T), order(T);
    for (int32_t j = 0; j < T; ++j) {
      double mc, qp;
      physical(t->sp, t->tx[j], t->tq[j], &mc, &qp);
      kc[j] = mbis::live_bins_m(mbis::total_mass_seconds(mc, qp), t->f_lo, t->df, K);
      order[j] = j;
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return kc[a] > kc[b]; });
    t->n_pass = (T + mbis::kPassTemplates - 1) / mbis::kPassTemplates;
    std::vector<int32_t> perm((size_t)t->n_pass * mbis::kPassTemplates, -1);
    t->nkb_pass.assign(t->n_pass, 0);
    for (int32_t i = 0; i < T; ++i) {
      perm[i] = order[i];
      const int32_t p = i / mbis::kPassTemplates;
      t->nkb_pass[p] = std::max(t->nkb_pass[p], (kc[order[i]] + mbis::kTileBins - 1) / mbis::kTileBins);
    }
    T_TRY(t, cudaMalloc(&t->d_perm, sizeof(int32_t) * perm.size()));
    T_TRY(t, cudaMemcpy(t->d_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));
    T_TRY(t, cudaMalloc(&t->d_tiles, (size_t)t->n_pass * t->n_kb * 2 * mbis::kTileBytes));
    T_TRY(t, mbis::launch_tiling_template_tiles(t->d_perm, t->n_pass, t->d_rows, g, t->d_tiles, nullptr));
    T_TRY(t, cudaDeviceSynchronize());
  }
  if (n_templates) *n_templates = t->T;
  if (n_used) *n_used = i;
  return MBIS_OK;
}

mbis_status mbis_tiling_templates(const mbis_tiling* t, int32_t* n_templates, double* coords, double* phys,
                                  int32_t* cand_index) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_templates: null tiling");
  if (n_templates) *n_templates = t->T;
  if (t->T == 0) return tfail(const_cast<mbis_tiling*>(t), MBIS_E_STATE, "mbis_tiling_templates: no bank");
  const int32_t T = t->T;
  for (int32_t j = 0; j < T; ++j) {
    if (coords) {
      coords[j] = t->tx[j];
      coords[T + j] = t->tq[j];
    }
    if (phys) physical(t->sp, t->tx[j], t->tq[j], &phys[j], &phys[T + j]);
    if (cand_index) cand_index[j] = t->cand_idx[j];
  }
  return MBIS_OK;
}

mbis_status mbis_tiling_match(mbis_tiling* t, int64_t n, const double* a, const double* b, double* out, void* stream) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_match: null tiling");
  if (n < 0 || (n > 0 && (!a || !b || !out))) return tfail(t, MBIS_E_INVALID, "mbis_tiling_match: bad n or buffer");
  T_TRY(t, mbis::launch_tiling_pair_match(t->sp, t->grid(), n, a, b, out, static_cast<cudaStream_t>(stream)));
  return MBIS_OK;
}

mbis_status mbis_tiling_assign(mbis_tiling* t, int64_t n, const double* pts, int32_t* tile, float* match, void* stream) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_assign: null tiling");
  if (t->T == 0) return tfail(t, MBIS_E_STATE, "mbis_tiling_assign: no bank");
  if (n < 0 || n > 2147483647LL || (n > 0 && (!pts || !tile)))
    return tfail(t, MBIS_E_INVALID, "mbis_tiling_assign: need 0 <= n < 2^31 and buffers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) return MBIS_OK;
  // process the points in order of their live-bin count, so that the 128 samples of a CTA
  // reach similar K (a stable counting sort on the count)
  if (n > t->scr_n) {
    drop_scratch(t);
    const int64_t n_seg = (n + mbis::kSortSegment - 1) / mbis::kSortSegment;
    if (cudaMalloc(&t->d_kc, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&t->d_rec, sizeof(float4) * 3 * n) != cudaSuccess ||
        cudaMalloc(&t->d_order, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&t->d_shist, sizeof(int32_t) * (size_t)n_seg * (t->K + 1)) != cudaSuccess ||
        cudaMalloc(&t->d_scount, sizeof(int32_t) * (t->K + 1)) != cudaSuccess ||
        cudaMalloc(&t->d_soffset, sizeof(int32_t) * (t->K + 1)) != cudaSuccess ||
        cudaMalloc(&t->d_snbad, sizeof(int32_t)) != cudaSuccess) {
      drop_scratch(t);
      return tfail(t, MBIS_E_OOM, "mbis_tiling_assign: out of device memory");
    }
    t->scr_n = n;
  }
  T_TRY(t, mbis::launch_tiling_setup(t->sp, t->grid(), n, pts, t->d_rec, t->d_kc, s));
  T_TRY(t, mbis::launch_tiling_lists(n, t->d_kc, t->K + 1, t->d_shist, t->d_scount, t->d_soffset, t->d_snbad,
                                     t->d_order, s));
  mbis::AssignArgs a;
  a.sp = t->sp;
  a.g = t->grid();
  a.n = n;
  a.rec = t->d_rec;
  a.order = t->d_order;
  a.tile = tile;
  a.match = match;
  a.T = t->T;
  a.n_pass = t->n_pass;
  a.perm = t->d_perm;
  a.tiles = static_cast<const unsigned char*>(t->d_tiles);
  a.bins = t->d_bins;
  a.err = t->d_err;
  for (int p = 0; p < mbis::kMaxPasses; ++p) a.nkb_pass[p] = p < t->n_pass ? t->nkb_pass[p] : 0;
  T_TRY(t, mbis::launch_tiling_assign(a, s));
  return MBIS_OK;
}

mbis_status mbis_tiling_set_pool(mbis_tiling* t, int64_t n, const double* pts, void* stream) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_set_pool: null tiling");
  if (t->T == 0) return tfail(t, MBIS_E_STATE, "mbis_tiling_set_pool: no bank");
  if (n < 1 || n > 2147483647LL || !pts) return tfail(t, MBIS_E_INVALID, "mbis_tiling_set_pool: need 1 <= n < 2^31");
  drop_pool(t);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n_seg = (n + mbis::kSortSegment - 1) / mbis::kSortSegment;
  const int32_t T = t->T;
  if (cudaMalloc(&t->d_pool, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&t->d_tile_of, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&t->d_members, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&t->d_hist, sizeof(int32_t) * (size_t)n_seg * T) != cudaSuccess ||
      cudaMalloc(&t->d_count, sizeof(int32_t) * T) != cudaSuccess ||
      cudaMalloc(&t->d_offset, sizeof(int32_t) * T) != cudaSuccess ||
      cudaMalloc(&t->d_nbad, sizeof(int32_t)) != cudaSuccess) {
    drop_pool(t);
    return tfail(t, MBIS_E_OOM, "mbis_tiling_set_pool: out of device memory");
  }
  t->N = n;
  T_TRY(t, cudaMemcpyAsync(t->d_pool, pts, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
  const mbis_status st = mbis_tiling_assign(t, n, t->d_pool, t->d_tile_of, nullptr, stream);
  if (st != MBIS_OK) {
    drop_pool(t);
    return st;
  }
  T_TRY(t, mbis::launch_tiling_lists(n, t->d_tile_of, T, t->d_hist, t->d_count, t->d_offset, t->d_nbad, t->d_members,
                                     s));
  T_TRY(t, cudaStreamSynchronize(s));
  int32_t errw = 0, nbad = 0;
  T_TRY(t, cudaMemcpy(&errw, t->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  T_TRY(t, cudaMemcpy(&nbad, t->d_nbad, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (errw != 0) {
    cudaMemset(t->d_err, 0, sizeof(int32_t));
    drop_pool(t);
    return tfail(t, MBIS_E_TIMEOUT, "mbis_tiling_set_pool: a device-side wait of the assignment timed out");
  }
  if (nbad != 0) {
    drop_pool(t);
    return tfail(t, MBIS_E_INVALID, "mbis_tiling_set_pool: " + std::to_string(nbad) + " pool points lie outside the space");
  }
  std::vector<int32_t> c32(T);
  T_TRY(t, cudaMemcpy(c32.data(), t->d_count, sizeof(int32_t) * T, cudaMemcpyDeviceToHost));
  t->counts.assign(c32.begin(), c32.end());
  return MBIS_OK;
}

mbis_status mbis_tiling_pool(const mbis_tiling* t, int64_t* counts, int32_t* tile_of, int32_t* members, void* stream) {
  mbis_tiling* tm = const_cast<mbis_tiling*>(t);
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_pool: null tiling");
  if (t->N == 0) return tfail(tm, MBIS_E_STATE, "mbis_tiling_pool: no pool");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (counts) std::copy(t->counts.begin(), t->counts.end(), counts);
  if (tile_of) T_TRY(tm, cudaMemcpyAsync(tile_of, t->d_tile_of, sizeof(int32_t) * t->N, cudaMemcpyDeviceToDevice, s));
  if (members) T_TRY(tm, cudaMemcpyAsync(members, t->d_members, sizeof(int32_t) * t->N, cudaMemcpyDeviceToDevice, s));
  return MBIS_OK;
}

mbis_status mbis_tiling_set_loglike(mbis_tiling* t, const double* ll, void* stream) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_set_loglike: null tiling");
  if (t->N == 0) return tfail(t, MBIS_E_STATE, "mbis_tiling_set_loglike: no pool");
  if (!ll) return tfail(t, MBIS_E_INVALID, "mbis_tiling_set_loglike: null log-likelihoods");
  drop_mixture(t);
  const int32_t T = t->T;
  if (cudaMalloc(&t->d_c, sizeof(double) * T) != cudaSuccess ||
      cudaMalloc(&t->d_mix, sizeof(double) * 2) != cudaSuccess ||
      cudaMalloc(&t->d_ll, sizeof(double) * T) != cudaSuccess ||
      cudaMalloc(&t->d_flag, sizeof(int32_t)) != cudaSuccess) {
    drop_mixture(t);
    return tfail(t, MBIS_E_OOM, "mbis_tiling_set_loglike: out of device memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  T_TRY(t, mbis::launch_tiling_mixture(T, t->d_count, ll, t->d_ll, t->d_c, t->d_mix, t->d_flag, s));
  T_TRY(t, cudaStreamSynchronize(s));
  int32_t flag = 1;
  T_TRY(t, cudaMemcpy(&flag, t->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (flag != 0) {
    drop_mixture(t);
    return tfail(t, MBIS_E_INVALID, "mbis_tiling_set_loglike: no tile with members has a finite log-likelihood");
  }
  t->has_mix = true;
  return MBIS_OK;
}

mbis_status mbis_tiling_draw(mbis_tiling* t, uint64_t seed, uint64_t ctr0, int64_t n, double* coords, double* theta,
                             double* log_q, double* log_prior, int32_t* pool_index, void* stream) {
  if (!t) return tfail(nullptr, MBIS_E_INVALID, "mbis_tiling_draw: null tiling");
  if (!t->has_mix) return tfail(t, MBIS_E_STATE, "mbis_tiling_draw: call mbis_tiling_set_loglike first");
  if (n < 0 || (n > 0 && (!theta || !log_q || !log_prior)))
    return tfail(t, MBIS_E_INVALID, "mbis_tiling_draw: bad n or null buffer");
  mbis::TilingDrawArgs a;
  a.sp = t->sp;
  a.seed = seed;
  a.ctr0 = ctr0;
  a.n = n;
  a.T = t->T;
  a.n_pool = t->N;
  a.pool = t->d_pool;
  a.count = t->d_count;
  a.offset = t->d_offset;
  a.members = t->d_members;
  a.c = t->d_c;
  a.mix = t->d_mix;
  a.ll = t->d_ll;
  a.log_prior = -std::log((t->sp.x_hi - t->sp.x_lo) * (t->sp.q_hi - t->sp.q_lo));
  a.coords = coords;
  a.theta = theta;
  a.log_q = log_q;
  a.log_p = log_prior;
  a.pool_index = pool_index;
  T_TRY(t, mbis::launch_tiling_draw(a, static_cast<cudaStream_t>(stream)));
  return MBIS_OK;
}

}  // extern "C"
