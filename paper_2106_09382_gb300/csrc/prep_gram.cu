// Data preparation (Section 2.1: columns centered; optionally scaled to unit
// 1/n variance) and the CUDA-core Gram S = Z^T Z / n (Algorithm 1's
// T <- X^T X, divided by n).
#include "prep_stats.h"
#include "fp_bits.cuh"

namespace concord {

template <typename TX>
__device__ __forceinline__ double ld_x(const TX* X, size_t i) {
  return to_f64(__ldg(X + i));
}

// One CTA per 32 columns; kStatThreads / 32 row groups per column sum
// disjoint row strides and are reduced in a fixed order, so the statistics
// are deterministic.  Two passes (mean, then centered sum of squares) in FP64.
constexpr int kStatThreads = 1024;

template <typename TX>
__global__ void __launch_bounds__(kStatThreads) k_col_stats(const TX* __restrict__ X, int n, int p,
                                                            int ldx, int prep,
                                                            double* __restrict__ mean,
                                                            double* __restrict__ inv_scale,
                                                            int* bad) {
  constexpr int G = kStatThreads / 32;  // row groups per column block
  __shared__ double part[G][33];
  __shared__ double s_mean[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + tx;
  double acc = 0.0;
  int nonfinite = 0;
  if (col < p) {
#pragma unroll 4
    for (int k = ty; k < n; k += G) {
      const double v = ld_x(X, (size_t)k * ldx + col);
      acc += v;
      if (!finite_bits(v)) nonfinite = 1;
    }
  }
  part[ty][tx] = acc;
  __syncthreads();
  if (ty == 0) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[g][tx];
    s_mean[tx] = (prep >= 1) ? s / n : 0.0;
  }
  __syncthreads();
  const double mu = s_mean[tx];
  acc = 0.0;
  if (col < p && prep == 2) {
#pragma unroll 4
    for (int k = ty; k < n; k += G) {
      const double d = ld_x(X, (size_t)k * ldx + col) - mu;
      acc += d * d;
    }
  }
  __syncthreads();
  part[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && col < p) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[g][tx];
    double inv = 1.0;
    if (prep == 2) {
      const double sd = sqrt(s / n);
      if (!(sd > 0.0)) atomicOr(bad, 1);
      inv = 1.0 / sd;
    }
    mean[col] = mu;
    inv_scale[col] = inv;
  }
  if (nonfinite) atomicOr(bad, 2);
}

// The same statistics over many CTAs: a CTA sums one chunk of rows for 128
// consecutive columns (coalesced across the CTA) into part[chunk * p + col];
// a second kernel adds the chunks of each column in chunk order (so the
// result is deterministic), then the centred sums of squares follow the same
// way.  Two passes, FP64, as the one-CTA-per-32-columns kernel above.
constexpr int kStatCols = 128;

template <typename TX, bool SQ>
__global__ void __launch_bounds__(kStatCols) k_col_partial(const TX* __restrict__ X, int n, int p,
                                                           int ldx, int rows_per_chunk,
                                                           const double* __restrict__ mean,
                                                           double* __restrict__ part,
                                                           int* __restrict__ bad) {
  const int col = blockIdx.x * kStatCols + threadIdx.x;
  if (col >= p) return;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(n, r0 + rows_per_chunk);
  const double mu = SQ ? mean[col] : 0.0;
  double acc = 0.0;
  int nonfinite = 0;
#pragma unroll 8
  for (int k = r0; k < r1; ++k) {
    const double v = ld_x(X, (size_t)k * ldx + col);
    if (SQ) {
      const double d = v - mu;
      acc += d * d;
    } else {
      acc += v;
      if (!finite_bits(v)) nonfinite = 1;
    }
  }
  part[(size_t)blockIdx.y * p + col] = acc;
  if (nonfinite) atomicOr(bad, 2);
}

// SQ = false: mean[col] (prep >= 1, else 0); SQ = true: inv_scale[col]
// (prep 2: 1 / population sd, flagging a constant column; else 1).
template <bool SQ>
__global__ void k_col_final(const double* __restrict__ part, int chunks, int n, int p, int prep,
                            double* __restrict__ mean, double* __restrict__ inv_scale,
                            int* __restrict__ bad) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= p) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[(size_t)c * p + col];
  if (!SQ) {
    mean[col] = prep >= 1 ? s / n : 0.0;
    if (prep < 2) inv_scale[col] = 1.0;
  } else {
    const double sd = sqrt(s / n);
    if (!(sd > 0.0)) atomicOr(bad, 1);
    inv_scale[col] = 1.0 / sd;
  }
}

template <typename TX, typename TZ>
__global__ void k_apply_prep(const TX* __restrict__ X, int n, int p, int ldx,
                             const double* __restrict__ mean, const double* __restrict__ inv_scale,
                             TZ* __restrict__ Z, int ldz) {
  const size_t total = (size_t)n * ldz;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ldz), i = (int)(e % ldz);
    Z[e] = (i < p) ? (TZ)((ld_x(X, (size_t)k * ldx + i) - mean[i]) * inv_scale[i]) : (TZ)0;
  }
}

cudaError_t launch_col_stats(const void* X, int x_f32, int n, int p, int ldx, int prep,
                             double* mean, double* inv_scale, int* bad, cudaStream_t st) {
  const int grid = (p + 31) / 32;
  if (x_f32)
    k_col_stats<float><<<grid, kStatThreads, 0, st>>>((const float*)X, n, p, ldx, prep, mean,
                                                      inv_scale, bad);
  else
    k_col_stats<double><<<grid, kStatThreads, 0, st>>>((const double*)X, n, p, ldx, prep, mean,
                                                       inv_scale, bad);
  note_launches(1);
  return cudaGetLastError();
}

int col_stats_chunks(int n) { return n < 32 ? n : 32; }

cudaError_t launch_col_stats_chunked(const void* X, int x_f32, int n, int p, int ldx, int prep,
                                     double* mean, double* inv_scale, int* bad, double* scratch,
                                     cudaStream_t st) {
  const int chunks = col_stats_chunks(n);
  const int rpc = (n + chunks - 1) / chunks;
  const dim3 grid((p + kStatCols - 1) / kStatCols, chunks);
  const int fg = (p + 255) / 256;
  if (x_f32)
    k_col_partial<float, false><<<grid, kStatCols, 0, st>>>((const float*)X, n, p, ldx, rpc, mean,
                                                            scratch, bad);
  else
    k_col_partial<double, false><<<grid, kStatCols, 0, st>>>((const double*)X, n, p, ldx, rpc, mean,
                                                             scratch, bad);
  k_col_final<false><<<fg, 256, 0, st>>>(scratch, chunks, n, p, prep, mean, inv_scale, bad);
  note_launches(2);
  if (prep == 2) {
    if (x_f32)
      k_col_partial<float, true><<<grid, kStatCols, 0, st>>>((const float*)X, n, p, ldx, rpc, mean,
                                                             scratch, bad);
    else
      k_col_partial<double, true><<<grid, kStatCols, 0, st>>>((const double*)X, n, p, ldx, rpc,
                                                              mean, scratch, bad);
    k_col_final<true><<<fg, 256, 0, st>>>(scratch, chunks, n, p, prep, mean, inv_scale, bad);
    note_launches(2);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_prep(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, void* Z, int z_f32, int ldz,
                              cudaStream_t st) {
  const int grid = 152 * 8;
  if (x_f32 && z_f32)
    k_apply_prep<float, float><<<grid, 256, 0, st>>>((const float*)X, n, p, ldx, mean, inv_scale,
                                                     (float*)Z, ldz);
  else if (x_f32)
    k_apply_prep<float, double><<<grid, 256, 0, st>>>((const float*)X, n, p, ldx, mean, inv_scale,
                                                      (double*)Z, ldz);
  else if (z_f32)
    k_apply_prep<double, float><<<grid, 256, 0, st>>>((const double*)X, n, p, ldx, mean, inv_scale,
                                                      (float*)Z, ldz);
  else
    k_apply_prep<double, double><<<grid, 256, 0, st>>>((const double*)X, n, p, ldx, mean,
                                                       inv_scale, (double*)Z, ldz);
  note_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S = Z^T Z * scale on CUDA cores.  64 x 64 output tiles of the upper
// triangle (tile row <= tile column), K chunks of 16 staged in shared memory,
// 16 x 16 threads with a 4 x 4 register block each (rows ty + 16 r, columns
// tx + 16 c).  Every tile is also written transposed, so S is exactly
// symmetric: (i, j) and (j, i) of a diagonal tile accumulate the same
// products in the same order.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_syrk(const T* __restrict__ Z, int n, int p, int ldz,
                                              T* __restrict__ S, int lds, T scale, int nb) {
  constexpr int BM = 64, BK = 16;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BM];
  // tile index -> (bi, bj), bi <= bj, row-major over the upper triangle
  int t = blockIdx.x, bi = 0;
  while (t >= nb - bi) {
    t -= nb - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = (T)0;
  for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int kk = idx >> 6, m = idx & 63;
      const int k = k0 + kk;
      const int ia = bi * BM + m, ib = bj * BM + m;
      As[kk][m] = (k < n && ia < p) ? Z[(size_t)k * ldz + ia] : (T)0;
      Bs[kk][m] = (k < n && ib < p) ? Z[(size_t)k * ldz + ib] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = bi * BM + ty + 16 * r, j = bj * BM + tx + 16 * c;
      if (i < p && j < p) {
        const T v = acc[r][c] * scale;
        S[(size_t)i * lds + j] = v;
        S[(size_t)j * lds + i] = v;
      }
    }
}

template <typename T>
static cudaError_t launch_syrk_t(const T* Z, int n, int p, int ldz, T* S, int lds, T scale,
                                 cudaStream_t st) {
  const int nb = (p + 63) / 64;
  const int tiles = nb * (nb + 1) / 2;
  k_syrk<T><<<tiles, 256, 0, st>>>(Z, n, p, ldz, S, lds, scale, nb);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_syrk_f64(const double* Z, int n, int p, int ldz, double* S, int lds, double scale,
                            cudaStream_t st) {
  return launch_syrk_t<double>(Z, n, p, ldz, S, lds, scale, st);
}
cudaError_t launch_syrk_f32(const float* Z, int n, int p, int ldz, float* S, int lds, float scale,
                            cudaStream_t st) {
  return launch_syrk_t<float>(Z, n, p, ldz, S, lds, scale, st);
}

}  // namespace concord
