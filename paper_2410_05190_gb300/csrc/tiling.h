// tiling.h -- device layout and kernel launchers of the tiled proposal (template bank,
// prior-volume tiles, mixture draws); not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mbis.h"

namespace mbis {

constexpr int kTileTemplates = 128;       // templates per MMA column block (N = 256 real columns)
constexpr int kPassTemplates = 2 * kTileTemplates;  // templates per pass of the assignment
constexpr int kTilingMaxTemplates = 16384;
constexpr int kMaxPasses = kTilingMaxTemplates / kPassTemplates;
constexpr int kBinRecord = 20;            // floats per bin pair of the FP32 table: 8 basis pairs, w pair, pad
constexpr int kTileBins = 32;             // bins per K-block of the assignment: 64 FP16 values, one 128-byte row
constexpr uint32_t kTileBytes = 32768;    // one half of a pass's K-block: 256 rows x 128 bytes

// The sampled space on the device.
struct TilingSpace {
  double x_lo, x_hi, mc_period, mc_base, q_lo, q_hi, chi1, chi2;
};

// Grid and noise weighting of the match.
struct TilingGrid {
  double f_lo, df;
  int32_t K;           // bins any point of the space reaches (largest live-bin count)
  int32_t n_kb;        // kTileBins-bin K-blocks covering K
  const double* w;     // [K] f^(-7/6) / sqrt(S)
  const double* w2sum; // [K + 1] prefix sums of w^2
  double wref;         // max w: the FP32 table holds w / wref
  double inv_wref2;    // 1 / wref^2
};

// FP64 unit-norm waveforms of n points (pts [2][n]): rows [n][K] (nullable) and k-major
// [K][ldk] (nullable, columns col0 .. col0 + n - 1).
cudaError_t launch_tiling_waveforms(const TilingSpace& sp, const TilingGrid& g, int32_t n, const double* pts,
                                    double2* rows, double2* kmaj, int32_t ldk, int32_t col0, cudaStream_t s);
// out[i][j] = |sum_k conj(A[i][k]) B[k][j]| for i < na, j < nb (FP64)
cudaError_t launch_tiling_absdots(int32_t na, const double2* A, int32_t nb, const double2* B, int32_t ldb, int32_t K,
                                  double* out, cudaStream_t s);
// FP64 match of n point pairs
cudaError_t launch_tiling_pair_match(const TilingSpace& sp, const TilingGrid& g, int64_t n, const double* a,
                                     const double* b, double* out, cudaStream_t s);
// copy rows src[idx[i]] (n rows of K) into dst rows row0 + i and k-major columns row0 + i
cudaError_t launch_tiling_append(int32_t n, const int32_t* idx, const double2* src, int32_t K, double2* dst_rows,
                                 int32_t row0, double2* dst_kmaj, int32_t ldk, cudaStream_t s);
// FP32 basis / weight records for the tensor-core pass: [n_kb * kTileBins / 2 bin pairs][kBinRecord]
cudaError_t launch_tiling_bin_records(const TilingGrid& g, double wscale, float* out, cudaStream_t s);
// FP16 template tiles: [n_pass][n_kb][2 halves][256 rows x 64] swizzled K-major, templates
// in the order perm ([n_pass * 256], -1 pads)
cudaError_t launch_tiling_template_tiles(const int32_t* perm, int32_t n_pass, const double2* rows, const TilingGrid& g,
                                         void* out, cudaStream_t s);
// set-up record of each point ([n][3] float4: FP32 phase coefficients, inverse norm,
// live-bin count; zero outside the space) and its live-bin count (the sort key)
cudaError_t launch_tiling_setup(const TilingSpace& sp, const TilingGrid& g, int64_t n, const double* pts, float4* rec,
                                int32_t* kc, cudaStream_t s);

struct AssignArgs {
  TilingSpace sp;
  TilingGrid g;
  int64_t n;
  const float4* rec;     // [n][3] set-up records
  const int32_t* order;  // [n] processing order of the points (null: as given)
  int32_t* tile;         // [n]
  float* match;          // [n] or null
  int32_t T, n_pass;
  const int32_t* perm;   // [n_pass * 256] template of each pass slot, -1 pads
  const unsigned char* tiles;  // FP16 template tiles
  const float* bins;     // bin records
  int32_t* err;          // device error word
  int32_t nkb_pass[kMaxPasses];  // K-blocks each pass's templates reach
};
cudaError_t launch_tiling_assign(const AssignArgs& a, cudaStream_t s);

// stable counting sort of tile indices into per-tile member lists
constexpr int kSortSegment = 8192;
cudaError_t launch_tiling_lists(int64_t n, const int32_t* tile, int32_t T, int32_t* hist /*[n_seg][T]*/,
                                int32_t* count, int32_t* offset, int32_t* n_bad, int32_t* members, cudaStream_t s);

// mixture: c[j] cumulative weights, mix = {m, total}; flag set when no tile can be drawn
cudaError_t launch_tiling_mixture(int32_t T, const int32_t* count, const double* ll, double* ll_copy, double* c,
                                  double* mix, int32_t* flag, cudaStream_t s);

struct TilingDrawArgs {
  TilingSpace sp;
  uint64_t seed, ctr0;
  int64_t n;
  int32_t T;
  int64_t n_pool;
  const double* pool;     // [2][n_pool]
  const int32_t* count;   // [T]
  const int32_t* offset;  // [T]
  const int32_t* members; // [n_pool]
  const double* c;        // [T]
  const double* mix;      // {m, total}
  const double* ll;       // [T]
  double log_prior;
  double* coords;         // [2][n] or null
  double* theta;          // [2][n]
  double* log_q;
  double* log_p;
  int32_t* pool_index;    // or null
};
cudaError_t launch_tiling_draw(const TilingDrawArgs& a, cudaStream_t s);

}  // namespace mbis
