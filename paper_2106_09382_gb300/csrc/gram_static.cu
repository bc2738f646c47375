// Gram without device allocation: S = Z^T Z / n in FP64 with the column
// statistics kept in a fixed device array of this file instead of memory
// allocated per call.
//
// Who needs it: callers that may not allocate device memory once they run.
// Examples are a host framework that owns all device memory through its own
// pool (a foreign cudaMalloc can fail against it or fragment it), a latency-
// critical loop where cudaMalloc / cudaFree would synchronise the device and
// stall other streams, and deployments that forbid dynamic allocation after
// start-up.  They pass X and S; the statistics live in g_gram_scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "concord.h"
#include "kernels.h"

namespace concord {

// Largest p the fixed array serves.
constexpr int kStaticGramMaxP = 16384;

// Fixed scratch, held by every device that loads the library until the
// process exits: column means [kStaticGramMaxP], inverse scales
// [kStaticGramMaxP], then one status word (as a double slot).  Every call
// shares it and it keeps the last call's contents; the status word is
// cleared at the start of each call.  Calls that overlap on the GPU (two
// streams, or two host threads at once) race on it.
static __device__ __align__(256) double g_gram_scratch[2 * kStaticGramMaxP + 32];

namespace {

// Device address of g_gram_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(CONCORD_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(CONCORD_E_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_gram_scratch);
    if (e != cudaSuccess || !ptr)
      return set_error(CONCORD_E_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                        : "cudaGetSymbolAddress gave NULL");
    g_scratch_addr[dev] = (double*)ptr;
  }
  *out = g_scratch_addr[dev];
  return CONCORD_OK;
}

// S = Z^T Z * scale with Z = (X - mean) * inv_scale formed while staging the
// tiles (no Z buffer): 64 x 64 upper-triangle output tiles, K chunks of 16,
// 16 x 16 threads with 4 x 4 register blocks, mirrored into the lower
// triangle.
template <typename TX>
__global__ void __launch_bounds__(256) k_syrk_std_f64(const TX* __restrict__ X, int n, int p, int ldx,
                                                      const double* __restrict__ mean,
                                                      const double* __restrict__ inv_scale,
                                                      double* __restrict__ S, int lds, double scale,
                                                      int nb) {
  constexpr int BM = 64, BK = 16;
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BM];
  int t = blockIdx.x, bi = 0;
  while (t >= nb - bi) {
    t -= nb - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int kk = idx >> 6, m = idx & 63;
      const int k = k0 + kk;
      const int ia = bi * BM + m, ib = bj * BM + m;
      As[kk][m] = (k < n && ia < p) ? ((double)X[(size_t)k * ldx + ia] - mean[ia]) * inv_scale[ia]
                                    : 0.0;
      Bs[kk][m] = (k < n && ib < p) ? ((double)X[(size_t)k * ldx + ib] - mean[ib]) * inv_scale[ib]
                                    : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double av[4], bv[4];
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
        const double v = acc[r][c] * scale;
        S[(size_t)i * lds + j] = v;
        S[(size_t)j * lds + i] = v;
      }
    }
}

}  // namespace
}  // namespace concord

using namespace concord;

extern "C" int concord_gram_static(const void* X_dev, int x_dtype, int n, int p, int ldx, int prep,
                                   double* S_dev, int lds, void* stream) {
  if (!X_dev || !S_dev || n < 1 || p < 2 || ldx < p || lds < p)
    return set_error(CONCORD_E_ARG, "X/S non-NULL, n >= 1, p >= 2, ldx >= p, lds >= p required");
  if (p > kStaticGramMaxP)
    return set_error(CONCORD_E_ARG,
                     "concord_gram_static serves p <= 16384 (its fixed scratch size); use "
                     "concord_gram for larger p");
  if ((x_dtype != CONCORD_F64 && x_dtype != CONCORD_F32) || prep < 0 || prep > 2)
    return set_error(CONCORD_E_ARG, "bad dtype or prep");
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != CONCORD_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  double* mean = scratch;
  double* inv = scratch + kStaticGramMaxP;
  int* bad = reinterpret_cast<int*>(scratch + 2 * kStaticGramMaxP);
  const int x_f32 = x_dtype == CONCORD_F32;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_col_stats(X_dev, x_f32, n, p, ldx, prep, mean, inv, bad, s);
  if (e == cudaSuccess) {
    const int nb = (p + 63) / 64;
    const int tiles = nb * (nb + 1) / 2;
    if (x_f32)
      k_syrk_std_f64<float><<<tiles, 256, 0, s>>>((const float*)X_dev, n, p, ldx, mean, inv, S_dev,
                                                  lds, 1.0 / n, nb);
    else
      k_syrk_std_f64<double><<<tiles, 256, 0, s>>>((const double*)X_dev, n, p, ldx, mean, inv,
                                                   S_dev, lds, 1.0 / n, nb);
    note_launches(1);
    e = cudaGetLastError();
  }
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(CONCORD_E_CUDA, cudaGetErrorString(e));
  if (hbad & 2) return set_error(CONCORD_E_NONFINITE, "X has a non-finite entry");
  if ((hbad & 1) && prep == CONCORD_PREP_STANDARDIZE)
    return set_error(CONCORD_E_NONPOS_DIAG, "X has a constant column");
  return CONCORD_OK;
}
