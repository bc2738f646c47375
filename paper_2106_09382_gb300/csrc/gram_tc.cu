// Tensor-core Gram for the mixed-precision path: S = Z^T Z / n from FP32
// operands split into tf32 hi + lo parts (3xTF32: hi*hi + hi*lo + lo*hi).
#include "kernels.h"

namespace concord {

__device__ __forceinline__ float to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Standardize, split and transpose: zt_hi[i * n_pad + k] = tf32(z_ki),
// zt_lo[i * n_pad + k] = tf32(z_ki - hi) with z = (x - mean_i) * inv_scale_i
// rounded to FP32.  32 x 32 tiles through shared memory; padding is zero.
template <typename TX>
__global__ void __launch_bounds__(256) k_split_tf32(const TX* __restrict__ X, int n, int p, int ldx,
                                                    const double* __restrict__ mean,
                                                    const double* __restrict__ inv_scale,
                                                    float* __restrict__ hi, float* __restrict__ lo,
                                                    int n_pad, int p_pad) {
  __shared__ float th[32][33];
  __shared__ float tl[32][33];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, i = i0 + tx;
    float z = 0.f;
    if (k < n && i < p) z = (float)(((double)X[(size_t)k * ldx + i] - mean[i]) * inv_scale[i]);
    const float h = to_tf32(z);
    th[r][tx] = h;
    tl[r][tx] = to_tf32(z - h);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i < p_pad && k < n_pad) {
      hi[(size_t)i * n_pad + k] = th[tx][r];
      lo[(size_t)i * n_pad + k] = tl[tx][r];
    }
  }
}

cudaError_t launch_split_tf32(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, float* zt_hi, float* zt_lo, int n_pad,
                              int p_pad, cudaStream_t st) {
  dim3 grid((n_pad + 31) / 32, (p_pad + 31) / 32);
  if (x_f32)
    k_split_tf32<float><<<grid, 256, 0, st>>>((const float*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                              zt_lo, n_pad, p_pad);
  else
    k_split_tf32<double><<<grid, 256, 0, st>>>((const double*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                               zt_lo, n_pad, p_pad);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram_tf32x3(const float*, const float*, int, int, int, float*, int, float,
                               cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace concord
