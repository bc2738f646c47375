// FP64-accurate S on the entries the solution depends on, for the FP64
// polish of a mixed-precision solve.
//
// Why: the tensor-core Gram (3xTF32 / 3xBF16) sums its products in the
// tensor cores' FP32 accumulators, which lose low bits in a biased way: on
// the AR(1) benchmark workload its diagonal is 1.1e-6 low on average, and
// the large off-diagonal entries are low by a similar relative amount.  A
// polish on that S finds the FP64 solution of a perturbed problem.  But the
// stationarity conditions of Eq. 1 on the active set read S only through
//   (Omega S)_ij + (Omega S)_ji  for active (i, j)  and  (Omega S)_ii,
// i.e. through s_kj with k in the support of row i and s_ki with k in the
// support of row j.  Recomputing exactly those entries (plus those of the
// pairs near the threshold, which decide the active set) makes the polish
// solve the exact problem; every other entry only enters the test
// |G_ij| <= lambda of pairs far below the threshold.
//
// Which entries: C is the candidate list of the next sweep (pairs with
// w_ij != 0 or |G_ij| > (1 - margin) lambda, i < j), N(i) the vertices paired
// with i in C.  For every candidate (i, j): s_kj for k in {i} u N(i) and s_ki
// for k in {j} u N(j); for every vertex i: s_ki for k in {i} u N(i).  Each
// entry is claimed once through a p x p bitmap (duplicates skip).
//
// How: z is the standardized data rounded to FP32 and stored transposed
// (zt: p_pad x ldn, one row per variable).  One warp computes one entry
// s_ab = sum_k z_ka z_kb / n: every lane sums its share of the products in
// double-float arithmetic (the exact product as hi + lo by an FMA, added with
// TwoSum into a (sum, compensation) pair), and the lanes' sums are combined
// in FP64.  The result differs from the FP64 Gram of the same data only
// through the FP32 rounding of z (random, relative 2^-24 per element).
#include "kernels.h"

namespace concord {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void k_nbr_count(const int2* __restrict__ cand, const int* __restrict__ n_cand,
                            int* __restrict__ cnt) {
  const int nc = *n_cand;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int2 e = cand[c];
    atomicAdd(cnt + e.x, 1);
    atomicAdd(cnt + e.y, 1);
  }
}

// off[i] = sum_{r < i} cnt[r] for i <= p; cur = off.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_nbr_scan(const int* __restrict__ cnt, int p,
                                                   int* __restrict__ off, int* __restrict__ cur) {
  __shared__ int s_warp[32];
  __shared__ int s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base <= p; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < p ? cnt[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const int excl = s_carry + (wid > 0 ? s_warp[wid - 1] : 0) + x - v;
    if (i <= p) {
      off[i] = excl;
      cur[i] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = excl + v;
    __syncthreads();
  }
}

__global__ void k_nbr_fill(const int2* __restrict__ cand, const int* __restrict__ n_cand,
                           int* __restrict__ cur, int* __restrict__ nbr) {
  const int nc = *n_cand;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int2 e = cand[c];
    nbr[atomicAdd(cur + e.x, 1)] = e.y;
    nbr[atomicAdd(cur + e.y, 1)] = e.x;
  }
}

// Pairs (i < j) of the dense iterate with w_ij != 0 or |W_ij + W_ji| > thr
// (used when no candidate list is at hand).  One warp per row.
__global__ void k_collect_dense(const float* __restrict__ Om, const float* __restrict__ W, int p,
                                int ld, float thr, int2* __restrict__ cand, int cap,
                                int* __restrict__ n_cand, int* __restrict__ dropped) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < p; i += warps) {
    for (int j0 = i + 1; j0 < p; j0 += 32) {
      const int j = j0 + lane;
      bool hit = false;
      if (j < p) {
        const float w = Om[(size_t)i * ld + j];
        hit = w != 0.f || fabsf(W[(size_t)i * ld + j] + W[(size_t)j * ld + i]) > thr;
      }
      const unsigned m = __ballot_sync(FULL, hit);
      if (!m) continue;
      int base = 0;
      if (lane == 0) base = atomicAdd(n_cand, __popc(m));
      base = __shfl_sync(FULL, base, 0);
      if (hit) {
        const int q = base + __popc(m & ((1u << lane) - 1u));
        if (q < cap)
          cand[q] = make_int2(i, j);
        else
          atomicAdd(dropped, 1);
      }
    }
  }
  // the list length is clamped by the consumers (min(n_cand, cap))
}

__global__ void k_clamp(int* __restrict__ n_cand, int cap) {
  if (*n_cand > cap) *n_cand = cap;
}

// Exact product of two floats as hi + lo (no contraction into an FMA of the
// product with a later add: __fmul_rn).
__device__ __forceinline__ void two_prod(float a, float b, float& hi, float& lo) {
  hi = __fmul_rn(a, b);
  lo = fmaf(a, b, -hi);
}

// (s, c) += x with TwoSum on s (the rounding error of s + x goes into c).
__device__ __forceinline__ void df_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, e);
}

// sum_k za[k] zb[k] over k < ldn (zero padded), by one warp; FP64 result in
// every lane.
__device__ __forceinline__ double warp_dot(const float* __restrict__ za,
                                           const float* __restrict__ zb, int ldn4, int lane) {
  float s = 0.f, c = 0.f;
  const float4* a4 = reinterpret_cast<const float4*>(za);
  const float4* b4 = reinterpret_cast<const float4*>(zb);
  for (int k = lane; k < ldn4; k += 32) {
    const float4 x = __ldg(a4 + k), y = __ldg(b4 + k);
    float h, l;
    two_prod(x.x, y.x, h, l);
    df_add(s, c, h);
    c = __fadd_rn(c, l);
    two_prod(x.y, y.y, h, l);
    df_add(s, c, h);
    c = __fadd_rn(c, l);
    two_prod(x.z, y.z, h, l);
    df_add(s, c, h);
    c = __fadd_rn(c, l);
    two_prod(x.w, y.w, h, l);
    df_add(s, c, h);
    c = __fadd_rn(c, l);
  }
  double v = (double)s + (double)c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// One warp per source: candidate c < nc gives the column groups (j; {i} u
// N(i)) and (i; {j} u N(j)); vertex source nc + i gives (i; {i} u N(i)).
__global__ void __launch_bounds__(256) k_refine(const int2* __restrict__ cand,
                                                const int* __restrict__ n_cand,
                                                const int* __restrict__ off,
                                                const int* __restrict__ nbr, int p,
                                                const float* __restrict__ zt, int ldn, double inv_n,
                                                double* __restrict__ S64, float* __restrict__ S32,
                                                int ld, unsigned* __restrict__ bitmap,
                                                float* __restrict__ mrow,
                                                int* __restrict__ n_done,
                                                int* __restrict__ ds_max) {
  const int lane = threadIdx.x & 31;
  const int nc = *n_cand;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int ldn4 = ldn >> 2;
  int done = 0;
  for (int src = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); src < nc + p; src += warps) {
    int cols[2], heads[2], groups;
    if (src < nc) {
      const int2 e = cand[src];
      cols[0] = e.y;  // s_kj for k in {i} u N(i)
      heads[0] = e.x;
      cols[1] = e.x;  // s_ki for k in {j} u N(j)
      heads[1] = e.y;
      groups = 2;
    } else {
      cols[0] = heads[0] = src - nc;  // s_ki for k in {i} u N(i)
      groups = 1;
    }
    for (int g = 0; g < groups; ++g) {
      const int col = cols[g], head = heads[g];
      const int b0 = off[head], b1 = off[head + 1];
      const float* zc = zt + (size_t)col * ldn;
      for (int t = b0 - 1; t < b1; ++t) {
        const int k = t < b0 ? head : nbr[t];
        const int a = k < col ? k : col, b = k < col ? col : k;
        const size_t bit = (size_t)a * p + b;
        unsigned claimed = 0;
        if (lane == 0) {
          const unsigned m = 1u << (bit & 31);
          claimed = (atomicOr(bitmap + (bit >> 5), m) & m) == 0u;
        }
        if (!__shfl_sync(FULL, claimed, 0)) continue;
        const double v = warp_dot(zt + (size_t)k * ldn, zc, ldn4, lane) * inv_n;
        if (lane == 0) {
          // the largest change of an entry against the FP32 S the sweeps so
          // far have used (float bits, rounded up; nonnegative floats order
          // as ints)
          const double dv = fabs(v - (double)S32[(size_t)a * ld + b]);
          if (dv > 0.0) atomicMax(ds_max, __float_as_int(nextafterf(__double2float_ru(dv), INFINITY)));
          S64[(size_t)a * ld + b] = v;
          S64[(size_t)b * ld + a] = v;
          S32[(size_t)a * ld + b] = (float)v;
          S32[(size_t)b * ld + a] = (float)v;
          if (a != b && mrow) {  // keep the row bounds valid (nonnegative floats order as ints)
            const int mb = __float_as_int(nextafterf(__double2float_ru(fabs(v)), INFINITY));
            atomicMax(reinterpret_cast<int*>(mrow) + a, mb);
            atomicMax(reinterpret_cast<int*>(mrow) + b, mb);
          }
          ++done;
        }
      }
    }
  }
  if (lane == 0 && done) atomicAdd(n_done, done);
}

}  // namespace

size_t refine_bitmap_words(int p) { return ((size_t)p * p + 31) / 32; }

cudaError_t launch_refine_s(const RefineArgs& a, cudaStream_t st) {
  const int p = a.p;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.bitmap, 0, sizeof(unsigned) * refine_bitmap_words(p), st))) return e;
  if ((e = cudaMemsetAsync(a.nbr_cnt, 0, sizeof(int) * (size_t)(p + 1), st))) return e;
  if ((e = cudaMemsetAsync(a.ctr, 0, sizeof(int) * kRefineCtrs, st))) return e;
  const int2* cand = a.cand;
  const int* n_cand = a.n_cand;
  if (!cand) {
    // no candidate list: collect the pairs from the dense FP32 iterate
    k_collect_dense<<<a.sms * 8, 256, 0, st>>>(a.Om32, a.W32, p, a.ld, a.thr, a.own_cand,
                                               a.own_cap, a.ctr + kRefineOwn,
                                               a.ctr + kRefineDropped);
    k_clamp<<<1, 1, 0, st>>>(a.ctr + kRefineOwn, a.own_cap);
    note_launches(2);
    cand = a.own_cand;
    n_cand = a.ctr + kRefineOwn;
  }
  k_nbr_count<<<a.sms * 4, 256, 0, st>>>(cand, n_cand, a.nbr_cnt);
  k_nbr_scan<<<1, 1024, 0, st>>>(a.nbr_cnt, p, a.nbr_off, a.nbr_cur);
  k_nbr_fill<<<a.sms * 4, 256, 0, st>>>(cand, n_cand, a.nbr_cur, a.nbr);
  k_refine<<<a.sms * 8, 256, 0, st>>>(cand, n_cand, a.nbr_off, a.nbr, p, a.zt, a.ldn,
                                      1.0 / a.n, a.S64, a.S32, a.ld, a.bitmap, a.mrow,
                                      a.ctr + kRefineDone, a.ctr + kRefineDs);
  note_launches(4);
  return cudaGetLastError();
}

}  // namespace concord
