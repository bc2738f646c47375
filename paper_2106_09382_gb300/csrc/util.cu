// Small elementwise / reduction kernels used around the sweep.
#include <atomic>

#include "kernels.h"
#include "fp_bits.cuh"

namespace concord {

static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, int ldi, TO* __restrict__ out, int ldo, int rows,
                          int cols) {
  const size_t total = (size_t)rows * ldo;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ldo), c = (int)(e % ldo);
    out[e] = (c < cols) ? (TO)in[(size_t)r * ldi + c] : (TO)0;
  }
}

cudaError_t launch_convert(const void* in, int in_f32, int ldi, void* out, int out_f32, int ldo,
                           int rows, int cols, cudaStream_t st) {
  const int grid = 152 * 8, block = 256;
  if (in_f32 && out_f32)
    k_convert<float, float><<<grid, block, 0, st>>>((const float*)in, ldi, (float*)out, ldo, rows,
                                                    cols);
  else if (in_f32)
    k_convert<float, double><<<grid, block, 0, st>>>((const float*)in, ldi, (double*)out, ldo, rows,
                                                     cols);
  else if (out_f32)
    k_convert<double, float><<<grid, block, 0, st>>>((const double*)in, ldi, (float*)out, ldo, rows,
                                                     cols);
  else
    k_convert<double, double><<<grid, block, 0, st>>>((const double*)in, ldi, (double*)out, ldo,
                                                      rows, cols);
  note_launches(1);
  return cudaGetLastError();
}

template <typename TA>
__global__ void k_extract_diag(const TA* __restrict__ A, int lda, int p, double* d64, float* d32,
                               double* dT64, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x) {
    const double v = (double)A[(size_t)i * lda + i];
    if (!isfinite(v))
      atomicOr(bad, 2);
    else if (!(v > 0.0))
      atomicOr(bad, 1);
    if (d64) d64[i] = v;
    if (d32) d32[i] = (float)v;
    if (dT64) dT64[i] = v;
  }
}

cudaError_t launch_extract_diag(const void* A, int a_f32, int lda, int p, double* d64, void* dT,
                                int t_f32, int* bad, cudaStream_t st) {
  const int grid = (p + 255) / 256;
  float* d32 = t_f32 ? (float*)dT : nullptr;
  double* dT64 = t_f32 ? nullptr : (double*)dT;
  if (a_f32)
    k_extract_diag<float><<<grid, 256, 0, st>>>((const float*)A, lda, p, d64, d32, dT64, bad);
  else
    k_extract_diag<double><<<grid, 256, 0, st>>>((const double*)A, lda, p, d64, d32, dT64, bad);
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_subdiag(const T* __restrict__ S, int ld, int p, int P, T* sd1, T* sd2) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p; v += gridDim.x * blockDim.x) {
    if (v == 0) {
      sd1[0] = (T)0;
      sd2[0] = (T)0;
      continue;
    }
    sd1[v] = S[(size_t)v * ld + (v - 1)];
    const int nx = (v >= 3) ? v - 2 : v - 2 + P;
    sd2[v] = (nx < p) ? S[(size_t)v * ld + nx] : (T)0;
  }
}

cudaError_t launch_subdiag(const void* S, int s_f32, int ld, int p, int P, void* sd1, void* sd2,
                           cudaStream_t st) {
  const int grid = (p + 255) / 256;
  if (s_f32)
    k_subdiag<float><<<grid, 256, 0, st>>>((const float*)S, ld, p, P, (float*)sd1, (float*)sd2);
  else
    k_subdiag<double><<<grid, 256, 0, st>>>((const double*)S, ld, p, P, (double*)sd1,
                                             (double*)sd2);
  note_launches(1);
  return cudaGetLastError();
}

// m[u] = an upper bound, as a float, of max_{x != u} |S[u][x]|: the exact
// maximum rounded up (for FP32 S also one float step above it, so that it
// bounds the FP64 copy of the same matrix as well).  One warp per row.
template <typename T>
__global__ void k_row_absmax(const T* __restrict__ S, int ld, int p, float* __restrict__ m) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < p; u += warps) {
    const T* row = S + (size_t)u * ld;
    T mx = (T)0;
    for (int x = lane; x < p; x += 32)
      if (x != u) mx = fmax(mx, fabs(row[x]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      float f;
      if (sizeof(T) == 4)
        f = nextafterf((float)mx, INFINITY);
      else
        f = __double2float_ru((double)mx);
      m[u] = f;
    }
  }
}

cudaError_t launch_row_absmax(const void* S, int s_f32, int ld, int p, float* m, cudaStream_t st) {
  const int grid = (p + 7) / 8 < 152 * 8 ? (p + 7) / 8 : 152 * 8;
  if (s_f32)
    k_row_absmax<float><<<grid, 256, 0, st>>>((const float*)S, ld, p, m);
  else
    k_row_absmax<double><<<grid, 256, 0, st>>>((const double*)S, ld, p, m);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void k_fill_f64(double* a, double v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

cudaError_t launch_fill_f64(double* a, double v, int n, cudaStream_t st) {
  k_fill_f64<<<(n + 255) / 256, 256, 0, st>>>(a, v, n);
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_set_identity(T* A, int p, int ld) {
  const size_t total = (size_t)p * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    A[e] = (r == c) ? (T)1 : (T)0;
  }
}

cudaError_t launch_set_identity(void* A, int a_f32, int p, int ld, cudaStream_t st) {
  if (a_f32)
    k_set_identity<float><<<152 * 8, 256, 0, st>>>((float*)A, p, ld);
  else
    k_set_identity<double><<<152 * 8, 256, 0, st>>>((double*)A, p, ld);
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_check_symmetric(const T* __restrict__ A, int p, int lda, int* bad) {
  const size_t total = (size_t)p * p;
  int flag = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / p), c = (int)(e % p);
    const T v = A[(size_t)r * lda + c];
    if (!isfinite((double)v)) flag |= 2;
    if (r < c && v != A[(size_t)c * lda + r]) flag |= 1;
  }
  if (flag) atomicOr(bad, flag);
}

cudaError_t launch_check_symmetric(const void* A, int a_f32, int p, int lda, int* bad,
                                   cudaStream_t st) {
  if (a_f32)
    k_check_symmetric<float><<<152 * 8, 256, 0, st>>>((const float*)A, p, lda, bad);
  else
    k_check_symmetric<double><<<152 * 8, 256, 0, st>>>((const double*)A, p, lda, bad);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void k_lambda_max(const double* __restrict__ S, int p, int ld, unsigned long long* out) {
  double m = 0.0;
  const size_t total = (size_t)p * p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    if (i < j) {
      const double v = fabs(S[(size_t)i * ld + j]) *
                       (1.0 / sqrt(S[(size_t)i * ld + i]) + 1.0 / sqrt(S[(size_t)j * ld + j]));
      m = fmax(m, v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_lambda_max(const double* S, int p, int ld, unsigned long long* out,
                              cudaStream_t st) {
  k_lambda_max<<<152 * 4, 256, 0, st>>>(S, p, ld, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace concord

// ---------------------------------------------------------------------------
// Helpers of the lambda path and stability selection.
// ---------------------------------------------------------------------------
namespace concord {
namespace {

template <typename TX>
__global__ void k_gather_rows(const TX* __restrict__ X, int ldx, const int* __restrict__ rows,
                              int nr, int p, double* __restrict__ out) {
  const size_t total = (size_t)nr * p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / p), c = (int)(e % p);
    out[e] = (double)X[(size_t)rows[r] * ldx + c];
  }
}

template <typename T>
__global__ void k_support_add(const T* __restrict__ Om, int ld, int p, float* __restrict__ cnt) {
  const size_t total = (size_t)p * p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / p), c = (int)(e % p);
    if (Om[(size_t)r * ld + c] != (T)0) atomicAdd(cnt + e, 1.0f);
  }
}

__global__ void k_scale_f32(float* a, size_t n, float s) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    a[e] *= s;
}

}  // namespace

cudaError_t launch_gather_rows(const void* X, int x_f32, int ldx, const int* rows, int nr, int p,
                               double* out, cudaStream_t st) {
  if (x_f32)
    k_gather_rows<float><<<152 * 4, 256, 0, st>>>((const float*)X, ldx, rows, nr, p, out);
  else
    k_gather_rows<double><<<152 * 4, 256, 0, st>>>((const double*)X, ldx, rows, nr, p, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_support_add(const void* Om, int f32, int ld, int p, float* cnt, cudaStream_t st) {
  if (f32)
    k_support_add<float><<<152 * 4, 256, 0, st>>>((const float*)Om, ld, p, cnt);
  else
    k_support_add<double><<<152 * 4, 256, 0, st>>>((const double*)Om, ld, p, cnt);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_f32(float* a, size_t n, float s, cudaStream_t st) {
  k_scale_f32<<<152 * 4, 256, 0, st>>>(a, n, s);
  note_launches(1);
  return cudaGetLastError();
}

// One warp per row u of S: 16-byte vectors of S in, of W, Omega and the FP64
// copy out; lane 0 then writes the row's scalars.
__global__ void __launch_bounds__(256) k_reset_mixed(const ResetMixedArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int nv = a.ld >> 2;  // float4 vectors per row (ld is a multiple of 32)
  for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < a.p; u += warps) {
    const float4* srow = reinterpret_cast<const float4*>(a.S + (size_t)u * a.ld);
    float4* wrow = reinterpret_cast<float4*>(a.W + (size_t)u * a.ld);
    float4* orow = reinterpret_cast<float4*>(a.Om + (size_t)u * a.ld);
    double2* drow = reinterpret_cast<double2*>(a.S64 + (size_t)u * a.ld);
    float mx = 0.f;
    // one pass over the row: the starting point's screen (upper triangle,
    // warp-uniform trips for the pushes), W = S, Omega = I, the FP64 copy
    for (int q0 = 0; q0 < nv; q0 += 32) {
      const int q = q0 + lane;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < nv) v = __ldg(srow + q);
      if (a.lam_s > 0.f) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = 4 * q + e;
          const float s = (&v.x)[e];
          const bool pred = q < nv && x > u && x < a.p && fabsf((0.f - s) - s) - a.lam_s > 0.f;
          const unsigned m = __ballot_sync(0xffffffffu, pred);
          if (!m) continue;
          int base = 0;
          if (lane == __ffs(m) - 1) base = atomicAdd(a.n_cand, __popc(m));
          base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
          if (pred) {
            const int r = base + __popc(m & ((1u << lane) - 1u));
            if (r < a.nc_cap) {  // a longer list is seen by its count
              a.cand[r] = make_int2(u, x);
              atomicAdd(a.cnt_r + u, 1);
              atomicAdd(a.cnt_r + x, 1);
            }
          }
        }
      }
      if (q < nv) {
        wrow[q] = v;
        const int c0 = 4 * q;
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u >= c0 && u < c0 + 4) (&o.x)[u - c0] = 1.f;
        orow[q] = o;
        drow[2 * q] = make_double2(widen_f32(v.x), widen_f32(v.y));
        drow[2 * q + 1] = make_double2(widen_f32(v.z), widen_f32(v.w));
        // padding columns are zero; the diagonal is left out
        if (c0 != u) mx = fmaxf(mx, fabsf(v.x));
        if (c0 + 1 != u) mx = fmaxf(mx, fabsf(v.y));
        if (c0 + 2 != u) mx = fmaxf(mx, fabsf(v.z));
        if (c0 + 3 != u) mx = fmaxf(mx, fabsf(v.w));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      const float* row = a.S + (size_t)u * a.ld;
      a.mrow[u] = nextafterf(mx, INFINITY);
      const float d = row[u];
      if (!isfinite(d))
        atomicOr(a.bad, 8);
      else if (!(d > 0.f))
        atomicOr(a.bad, 16);
      a.sdiag64[u] = (double)d;
      a.sdiag32[u] = d;
      a.omdiag64[u] = 1.0;
      float s1 = 0.f, s2 = 0.f;
      if (u > 0) {
        s1 = row[u - 1];
        const int nx = (u >= 3) ? u - 2 : u - 2 + a.P;
        s2 = nx < a.p ? row[nx] : 0.f;
      }
      a.sd1[u] = s1;
      a.sd2[u] = s2;
      a.sd1_64[u] = (double)s1;
      a.sd2_64[u] = (double)s2;
    }
  }
}

cudaError_t launch_reset_mixed(const ResetMixedArgs& a, cudaStream_t st) {
  const int grid = (a.p + 7) / 8 < 152 * 8 ? (a.p + 7) / 8 : 152 * 8;
  k_reset_mixed<<<grid, 256, 0, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace concord
