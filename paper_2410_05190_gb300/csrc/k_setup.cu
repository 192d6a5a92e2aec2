// k_setup.cu -- per-event table kernels (FP64), run once per event at set-up.
//
// For each bin k and detector d the data enter the likelihood only through
//   c_dk = 4 df conj(d_dk) f_k^(-7/6) / S_dk          (Eq. 1 with the f^(-7/6) amplitude)
//   w_dk = 4 df f_k^(-7/3) / S_dk                       (the <h|h> integrand per unit A^2)
// so (d|h)_d = Re(A P_d sum_k c_dk e^(-i (Psi_k + 2 pi f_k dt_d))) and
// (h|h)_d = A^2 |P_d|^2 sum_{k < k_cut} w_dk (Eqs. 1-3).  When sky position, polarisation and
// inclination are fixed for the event, P_d and dt_d are constants and the detectors fold
// into one table C_k = sum_d P_d c_dk e^(-2 pi i f_k dt_d) and one weight W_k.
#include "internal.h"

namespace mbis {
namespace {

__global__ void basis_table_kernel(double f_lo, double df, int32_t n, double* out) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double f = f_lo + (double)k * df;
#pragma unroll
  for (int j = 0; j < kNumBasis; ++j) out[(int64_t)j * n + k] = basis(j, f);
}

struct DetPack {
  DetResponse d[kMaxDet];
};

__global__ void event_tables_kernel(int32_t n_det, int32_t n, double f_lo, double df, int32_t dtype,
                                    const void* strain, const double* psd, int32_t fold, DetPack det, double2* c_out,
                                    double* w_out) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double f = f_lo + (double)k * df;
  const double amp = pow(f, -7.0 / 6.0);
  double cr = 0.0, ci = 0.0, wsum = 0.0;
  for (int d = 0; d < n_det; ++d) {
    const int64_t idx = (int64_t)d * n + k;
    double dr, di;
    if (dtype == MBIS_C128) {
      const double2 v = reinterpret_cast<const double2*>(strain)[idx];
      dr = v.x; di = v.y;
    } else {
      const float2 v = reinterpret_cast<const float2*>(strain)[idx];
      dr = v.x; di = v.y;
    }
    const double S = psd[idx];
    const double g = 4.0 * df * amp / S;
    const double xr = g * dr, xi = -g * di;  // c_dk
    const double wt = 4.0 * df * amp * amp / S;
    if (fold) {
      double s, c;
      sincospi(2.0 * f * det.d[d].dt, &s, &c);  // e^(-2 pi i f dt) = c - i s
      const double er = c, ei = -s;
      const double yr = xr * er - xi * ei, yi = xr * ei + xi * er;
      cr += det.d[d].pre * yr - det.d[d].pim * yi;
      ci += det.d[d].pre * yi + det.d[d].pim * yr;
      wsum += (det.d[d].pre * det.d[d].pre + det.d[d].pim * det.d[d].pim) * wt;
    } else {
      c_out[idx] = make_double2(xr, xi);
      w_out[idx] = wt;
    }
  }
  if (fold) {
    c_out[k] = make_double2(cr, ci);
    w_out[k] = wsum;
  }
}

// One block per row: T[r][0] = 0, T[r][k + 1] = T[r][k] + w[r][k], in a fixed order.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) prefix_rows_kernel(const double* w, int32_t n, double* T) {
  __shared__ double part[kScanThreads];
  const double* wr = w + (int64_t)blockIdx.x * n;
  double* Tr = T + (int64_t)blockIdx.x * (n + 1);
  const int32_t per = (n + kScanThreads - 1) / kScanThreads;
  const int32_t a = threadIdx.x * per, b = min(n, a + per);
  double s = 0.0;
  for (int32_t k = a; k < b; ++k) s += wr[k];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {  // sequential exclusive scan of the 1024 partial sums
    double run = 0.0;
    for (int i = 0; i < kScanThreads; ++i) {
      const double v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  double run = part[threadIdx.x];
  if (threadIdx.x == 0) Tr[0] = 0.0;
  for (int32_t k = a; k < b; ++k) {
    run += wr[k];
    Tr[k + 1] = run;
  }
}

__global__ void max_abs_kernel(const double2* c, int32_t n, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int32_t k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, hypot(c[k].x, c[k].y));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// FP32 table in bin pairs: (re_k, re_k+1, im_k, im_k+1) for even k, zero past n
__global__ void to_f32_kernel(const double2* c, int32_t n, int32_t n_pad, double inv_scale, float4* out) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n_pad) return;
  const int32_t k = 2 * p;
  const double2 a = k < n ? c[k] : make_double2(0.0, 0.0);
  const double2 b = k + 1 < n ? c[k + 1] : make_double2(0.0, 0.0);
  out[p] = make_float4((float)(a.x * inv_scale), (float)(b.x * inv_scale), (float)(a.y * inv_scale),
                       (float)(b.y * inv_scale));
}

// e^(-2 pi i f_k tau_j) as (cos, sin) of 2 pi f_k tau_j, tau_j = (j - J/2) dt: [n][J]
__global__ void twiddle_kernel(int32_t n, double f_lo, double df, int32_t J, double dt, double2* out) {
  const int32_t k = blockIdx.x;
  for (int32_t j = threadIdx.x; j < J; j += blockDim.x) {
    const double f = f_lo + (double)k * df, tau = (double)(j - J / 2) * dt;
    double s, c;
    sincospi(2.0 * f * tau, &s, &c);
    out[(int64_t)k * J + j] = make_double2(c, s);
  }
}

// per-detector FP32 tables, scaled, zero-padded to n_pad: [rows][n_pad]
// rows of n complex values -> FP32, padded to n_pad (even) bins, bin pairs interleaved as
// (re_k, re_k+1, im_k, im_k+1) so that a pair loads as one 16-byte vector of two f32x2 lanes
__global__ void rows_to_f32_kernel(const double2* c, int32_t rows, int32_t n, int32_t n_pad, double inv_scale,
                                   float2* out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t r = blockIdx.y;
  if (k >= n_pad || r >= rows) return;
  const double2 v = k < n ? c[(int64_t)r * n + k] : make_double2(0.0, 0.0);
  float* row = reinterpret_cast<float*>(out + (int64_t)r * n_pad);
  const int32_t p = k >> 1, e = k & 1;
  row[4 * p + e] = (float)(v.x * inv_scale);
  row[4 * p + 2 + e] = (float)(v.y * inv_scale);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// Twiddle operand of the time-shift contraction, one 16-bin K-block per CTA, one shift per
// thread: row j holds (cos, sin)(2 pi f_k tau_j) for the block's 16 bins, split into a TF32
// head and a tail (the remainder, rounded to TF32 as well), each in the 128-byte-swizzled
// K-major layout that the tensor core
// reads (16-byte chunk c of row j at byte j*128 + ((c ^ (j & 7)) << 4)).
// out: [n_kb][2 (head, tail)][128 rows x 128 bytes].
__global__ void twiddle_tiles_kernel(int32_t n, double f_lo, double df, double dt, int32_t n_kb, float* out) {
  const int32_t kb = blockIdx.x, j = threadIdx.x;
  if (kb >= n_kb || j >= 128) return;
  const double tau = (double)(j - 64) * dt;
  float* head = out + (int64_t)kb * 2 * 4096;
  float* tail = head + 4096;
  for (int kk = 0; kk < 16; ++kk) {
    const int32_t k = 16 * kb + kk;
    double s = 0.0, c = 0.0;
    if (k < n) sincospi(2.0 * (f_lo + (double)k * df) * tau, &s, &c);
    const float v[2] = {(float)c, (float)s};
    for (int e = 0; e < 2; ++e) {
      const int kidx = 2 * kk + e;  // K index inside the block
      const int chunk = kidx >> 2, pos = kidx & 3;
      const int word = j * 32 + (((chunk ^ (j & 7)) << 2) | pos);
      const float h = tf32_round(v[e]);
      head[word] = h;
      tail[word] = tf32_round(v[e] - h);  // the tensor core would truncate an unrounded tail
    }
  }
}

}  // namespace

cudaError_t launch_rows_to_f32(const double2* c, int32_t rows, int32_t n, int32_t n_pad, double inv_scale,
                               float2* out, cudaStream_t s) {
  dim3 grid((n_pad + 255) / 256, rows);
  rows_to_f32_kernel<<<grid, 256, 0, s>>>(c, rows, n, n_pad, inv_scale, out);
  return cudaGetLastError();
}

cudaError_t launch_twiddle_tiles(int32_t n, double f_lo, double df, double dt, int32_t n_kb, float* out,
                                 cudaStream_t s) {
  twiddle_tiles_kernel<<<n_kb, 128, 0, s>>>(n, f_lo, df, dt, n_kb, out);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(int32_t n, double f_lo, double df, int32_t J, double dt, double2* out, cudaStream_t s) {
  twiddle_kernel<<<n, 128, 0, s>>>(n, f_lo, df, J, dt, out);
  return cudaGetLastError();
}

cudaError_t launch_basis_table(double f_lo, double df, int32_t n, double* out, cudaStream_t s) {
  basis_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(f_lo, df, n, out);
  return cudaGetLastError();
}

cudaError_t launch_event_tables(int32_t n_det, int32_t n_bins, double f_lo, double df, int32_t dtype,
                                const void* strain, const double* psd, int32_t fold, const DetResponse* det,
                                double2* c_out, double* w_out, cudaStream_t s) {
  DetPack p = {};
  if (det != nullptr)  // the per-detector tables (fold = 0) take no responses
    for (int d = 0; d < n_det && d < kMaxDet; ++d) p.d[d] = det[d];
  event_tables_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(n_det, n_bins, f_lo, df, dtype, strain, psd, fold, p,
                                                            c_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_prefix_rows(const double* w, int32_t rows, int32_t n, double* T, cudaStream_t s) {
  prefix_rows_kernel<<<rows, kScanThreads, 0, s>>>(w, n, T);
  return cudaGetLastError();
}

cudaError_t launch_max_abs(const double2* c, int32_t n, double* out, cudaStream_t s) {
  max_abs_kernel<<<1, 256, 0, s>>>(c, n, out);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double2* c, int32_t n, int32_t n_pad, double inv_scale, float4* out, cudaStream_t s) {
  to_f32_kernel<<<(n_pad / 2 + 255) / 256, 256, 0, s>>>(c, n, n_pad, inv_scale, out);
  return cudaGetLastError();
}

}  // namespace mbis
