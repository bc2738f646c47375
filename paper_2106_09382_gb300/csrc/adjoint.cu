// Implicit differentiation of the CONCORD estimate on its active set.
//
// At a minimiser of Eq. 1 (S units) the subgradient conditions hold with
// equality on the active set A (the diagonal and the pairs w_ij != 0):
//   F_ii = W_ii - 1 / w_ii = 0,   F_ij = W_ij + W_ji + lambda sign(w_ij) = 0,
// W = Omega S.  With A and the signs locally fixed, the implicit-function
// theorem gives d Omega_A = -H^{-1} dF with H the Hessian of the smooth part
// of Eq. 1 on A: for a symmetric direction V supported on A,
//   (H V)_ij = (V S)_ij + (V S)_ji,   (H V)_ii = (V S)_ii + v_ii / w_ii^2.
// A loss gradient b on A gives the adjoint a = H^{-1} b (preconditioned
// conjugate gradients, one persistent cooperative launch), and from it
//   dL/dlambda = -sum_{i<j in A} a_ij sign(w_ij),   dL/dS = -Omega Ahat,
// and dL/dX through S = Z^T Z / n and the data preparation of Section 2.1.
//
// Layout: A is held as CSR rows N(i) + {i} with sorted columns (both
// orientations of every pair, the diagonal included).  Every vector of the
// iteration (b, a, r, z, p, H p) lives on the CSR entries with the two
// orientations of a pair holding the same value; entry e's partner (j, i) is
// mirror[e].  A product (V S)_ij for an entry (i, j) is a gather of row j of S
// at the columns of N(i) + {i}: one warp per upper entry (j >= i) sums both
// orientations and writes the pair's two slots.  S is FP64 and read-only
// (L2-resident at the sizes of interest).
#include <math.h>

#include "adjoint.h"

namespace concord {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Per-CTA sums of K per-thread values, in a fixed order (warps, then lanes by
// a shuffle tree), written by thread 0 to out[k].
template <int K>
__device__ void block_sums(const double (&v)[K], double* out) {
  __shared__ double red[32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s[k] = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp][k] = s[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w][k];
      out[k] = t;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- active set

template <typename T>
__global__ void k_adj_count(const T* __restrict__ Om, int p, int ld, int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < p; i += nw) {
    const T* row = Om + (size_t)i * ld;
    int c = 0;
    for (int j = lane; j < p; j += 32) c += (row[j] != T(0) || j == i) ? 1 : 0;
    c = warp_sum_int(c);
    if (lane == 0) cnt[i] = c;
  }
}

// rowptr[0] = 0, rowptr[i + 1] = rowptr[i] + cnt[i]  (one CTA).
__global__ void k_adj_scan(const int* __restrict__ cnt, int p, int* __restrict__ rowptr) {
  __shared__ int ws[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    carry = 0;
    rowptr[0] = 0;
  }
  __syncthreads();
  for (int base = 0; base < p; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int x = i < p ? cnt[i] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < nw ? ws[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const int incl = carry + (warp ? ws[warp - 1] : 0) + x;
    if (i < p) rowptr[i + 1] = incl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
}

template <typename T>
__global__ void k_adj_fill(const T* __restrict__ Om, int p, int ld, const int* __restrict__ rowptr,
                           int* __restrict__ col, int* __restrict__ erow, double* __restrict__ om) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < p; i += nw) {
    const T* row = Om + (size_t)i * ld;
    int base = rowptr[i];
    for (int j0 = 0; j0 < p; j0 += 32) {
      const int j = j0 + lane;
      T v = T(0);
      bool nz = false;
      if (j < p) {
        v = row[j];
        nz = (v != T(0)) || j == i;
      }
      const unsigned m = __ballot_sync(0xffffffffu, nz);
      if (nz) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        col[pos] = j;
        erow[pos] = i;
        om[pos] = (double)v;
      }
      base += __popc(m);
    }
  }
}

// mirror[e] = the entry (j, i) of entry e = (i, j); minv[e] = 1 / H_ee
// (Jacobi preconditioner: s_ii + 1/w_ii^2 on the diagonal, s_ii + s_jj on a
// pair).  bad = 1 if a pair has no partner (Omega not symmetric) or the
// diagonal is not positive.
__global__ void k_adj_prep(int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const int* __restrict__ erow, const double* __restrict__ om,
                           const double* __restrict__ sdiag, int* __restrict__ mirror,
                           double* __restrict__ minv, int* __restrict__ bad) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
    const int i = erow[e], j = col[e];
    if (i == j) {
      mirror[e] = e;
      const double w = om[e];
      if (!(w > 0.0)) atomicOr(bad, 1);
      minv[e] = 1.0 / (sdiag[i] + 1.0 / (w * w));
      continue;
    }
    int lo = rowptr[j], hi = rowptr[j + 1] - 1, m = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = col[mid];
      if (c == i) {
        m = mid;
        break;
      }
      if (c < i) lo = mid + 1;
      else hi = mid - 1;
    }
    if (m < 0 || om[m] != om[e]) atomicOr(bad, 1);
    mirror[e] = m < 0 ? e : m;
    minv[e] = 1.0 / (sdiag[i] + sdiag[j]);
  }
}

// b on A from a dense loss gradient (full-matrix convention).
template <typename G>
__global__ void k_adj_rhs_dense(const G* __restrict__ g, int ldg, int nnz, const int* __restrict__ col,
                                const int* __restrict__ erow, double* __restrict__ b) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
    const int i = erow[e], j = col[e];
    const double gij = (double)g[(size_t)i * ldg + j];
    b[e] = (i == j) ? gij : gij + (double)g[(size_t)j * ldg + i];
  }
}

// Lane-strided partial of sum_{t in row a} v(t) M[b, col[t]]  (not reduced).
template <typename M, typename VF>
__device__ __forceinline__ double gather_row(int a, int b, const int* __restrict__ rowptr,
                                             const int* __restrict__ col, const M* __restrict__ Mx,
                                             int ldm, VF v, int lane) {
  const M* mrow = Mx + (size_t)b * ldm;
  double s = 0.0;
  const int t1 = rowptr[a + 1];
  for (int t = rowptr[a] + lane; t < t1; t += 32) s = fma(v(t), (double)__ldg(mrow + col[t]), s);
  return s;
}

// Held-out loss and its gradient on A: with R = Omega S_val,
//   b_ii = R_ii - 1/w_ii,  b_ij = R_ij + R_ji,
//   loss = -sum log w_ii + 1/2 (sum_i R_ii w_ii + sum_{i<j} w_ij (R_ij + R_ji)).
// One warp per upper entry; per-CTA loss partials in part[blockIdx.x].
template <typename M>
__global__ void k_adj_heldout(int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                              const int* __restrict__ erow, const int* __restrict__ mirror,
                              const double* __restrict__ om, const M* __restrict__ Sv, int lds,
                              double* __restrict__ b, double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  auto v = [&](int t) { return om[t]; };
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nnz; e += nw) {
    const int i = erow[e], j = col[e];
    if (j < i) continue;
    double s = gather_row(i, j, rowptr, col, Sv, lds, v, lane);
    if (i != j) s += gather_row(j, i, rowptr, col, Sv, lds, v, lane);
    s = warp_sum(s);
    if (lane == 0) {
      const double w = om[e];
      if (i == j) {
        b[e] = s - 1.0 / w;
        acc += 0.5 * s * w - log(w);
      } else {
        b[e] = s;
        b[mirror[e]] = s;
        acc += 0.5 * w * s;
      }
    }
  }
  double vals[1] = {acc};
  block_sums<1>(vals, part + blockIdx.x);
}

// out[0] = sum of part[0..n) in order (one warp).
__global__ void k_adj_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s += part[k];
  s = warp_sum(s);
  if (lane == 0) out[0] = s;
}

// ---------------------------------------------------------------- PCG
template <int K>
__device__ __forceinline__ void grid_sums(const double* part, int slot0, double (&out)[K]) {
  // every CTA sums the same partials in the same order
  __shared__ double sh[K];
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = 0.0;
      for (int g = threadIdx.x; g < (int)gridDim.x; g += 32) s += part[g * kParts + slot0 + q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) sh[q] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = sh[q];
  __syncthreads();
}

__device__ __forceinline__ bool aborted(const WaitCtl& w) {
  return *(volatile int*)w.abort != 0;
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_cg(const AdjArgs a) {
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int gw = tid >> 5, nw = nthr >> 5;
  const int nnz = a.nnz;
  double* part = a.partials + (size_t)blockIdx.x * kParts;
  unsigned gen = 0;

  // x = 0, r = b, z = M^-1 b, p = 0
  {
    double rz = 0.0, rr = 0.0;
    for (int e = tid; e < nnz; e += nthr) {
      const double bv = a.b[e];
      const double zv = a.minv[e] * bv;
      a.x[e] = 0.0;
      a.r[e] = bv;
      a.z[e] = zv;
      a.pb0[e] = 0.0;
      if (a.col[e] >= a.erow[e]) {
        rz = fma(bv, zv, rz);
        rr = fma(bv, bv, rr);
      }
    }
    double vals[2] = {rz, rr};
    block_sums<2>(vals, part + kAdjPartRz);
  }
  grid_barrier(a.barrier, gen, a.wait, 0);
  if (aborted(a.wait)) return;
  double sums[2];
  grid_sums<2>(a.partials, kAdjPartRz, sums);
  double rz = sums[0], rr = sums[1];
  const double bb = rr;
  const double stop = a.tol * a.tol * bb;
  int status = (bb == 0.0) ? 0 : 1;
  int it = 0;
  double rz_prev = 1.0;
  double* pold = a.pb0;
  double* pnew = a.pb1;
  for (; status == 1 && it < a.max_iter; ++it) {
    if (rr <= stop) {
      status = 0;
      break;
    }
    const double beta = it ? rz / rz_prev : 0.0;
    // phase A: p = z + beta p_old (formed where it is read), q = H p, <p, q>
    double ppq = 0.0;
    {
      const double* z = a.z;
      const double* po = pold;
      auto v = [&](int t) { return fma(beta, po[t], z[t]); };
      for (int e = gw; e < nnz; e += nw) {
        const int i = a.erow[e], j = a.col[e];
        if (j < i) continue;
        double s = gather_row(i, j, a.rowptr, a.col, a.S, a.ld, v, lane);
        if (i != j) s += gather_row(j, i, a.rowptr, a.col, a.S, a.ld, v, lane);
        s = warp_sum(s);
        if (lane == 0) {
          const double pe = v(e);
          if (i == j) {
            const double w = a.om[e];
            s += pe / (w * w);
          } else {
            const int m = a.mirror[e];
            a.q[m] = s;
            pnew[m] = pe;
          }
          a.q[e] = s;
          pnew[e] = pe;
          ppq = fma(pe, s, ppq);
        }
      }
    }
    {
      double vals[1] = {ppq};
      block_sums<1>(vals, part + kAdjPartPq);
    }
    grid_barrier(a.barrier, gen, a.wait, 1);
    if (aborted(a.wait)) return;
    double pqs[1];
    grid_sums<1>(a.partials, kAdjPartPq, pqs);
    const double pq = pqs[0];
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = 2;  // H not positive definite along p, or non-finite
      break;
    }
    const double alpha = rz / pq;
    // phase B: x += alpha p, r -= alpha q, z = M^-1 r
    double prz = 0.0, prr = 0.0;
    for (int e = tid; e < nnz; e += nthr) {
      const int i = a.erow[e], j = a.col[e];
      if (j < i) continue;
      const double pe = pnew[e], qe = a.q[e];
      const double xe = fma(alpha, pe, a.x[e]);
      const double re = fma(-alpha, qe, a.r[e]);
      const double ze = a.minv[e] * re;
      a.x[e] = xe;
      a.r[e] = re;
      a.z[e] = ze;
      if (i != j) {
        const int m = a.mirror[e];
        a.x[m] = xe;
        a.r[m] = re;
        a.z[m] = ze;
      }
      prz = fma(re, ze, prz);
      prr = fma(re, re, prr);
    }
    {
      double vals[2] = {prz, prr};
      block_sums<2>(vals, part + kAdjPartRz);
    }
    grid_barrier(a.barrier, gen, a.wait, 2);
    if (aborted(a.wait)) return;
    grid_sums<2>(a.partials, kAdjPartRz, sums);
    rz_prev = rz;
    rz = sums[0];
    rr = sums[1];
    double* t = pold;
    pold = pnew;
    pnew = t;
  }
  if (status == 1 && rr <= stop) status = 0;

  // epilogue: true residual ||b - H x||^2 and dL/dlambda = -sum_pairs x sign(w)
  {
    double res = 0.0, dl = 0.0;
    const double* x = a.x;
    auto v = [&](int t) { return x[t]; };
    for (int e = gw; e < nnz; e += nw) {
      const int i = a.erow[e], j = a.col[e];
      if (j < i) continue;
      double s = gather_row(i, j, a.rowptr, a.col, a.S, a.ld, v, lane);
      if (i != j) s += gather_row(j, i, a.rowptr, a.col, a.S, a.ld, v, lane);
      s = warp_sum(s);
      if (lane == 0) {
        const double w = a.om[e];
        if (i == j) s += x[e] / (w * w);
        else dl -= (w > 0.0 ? x[e] : -x[e]);
        const double d = a.b[e] - s;
        res = fma(d, d, res);
      }
    }
    double vals[2] = {res, dl};
    block_sums<2>(vals, part + kAdjPartRes);
  }
  grid_barrier(a.barrier, gen, a.wait, 3);
  if (aborted(a.wait)) return;
  if (blockIdx.x == 0) {
    double fin[2];
    grid_sums<2>(a.partials, kAdjPartRes, fin);
    if (threadIdx.x == 0) {
      a.result[kAdjIters] = it;
      a.result[kAdjRel] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      a.result[kAdjTrue] = bb > 0.0 ? sqrt(fin[0] / bb) : 0.0;
      a.result[kAdjDlam] = fin[1];
      a.result[kAdjStatus] = status;
      a.result[kAdjBnorm] = sqrt(bb);
    }
  }
}

// ---------------------------------------------------------------- dL/dS
// out (p x ldo, FP64) = -Omega Ahat: row i = -sum_{k in N(i)+{i}} w_ik Ahat_k.
// One warp per row: the row is zeroed, then each term adds a sparse row of
// Ahat (distinct columns per term; the warp's terms run in order).
__global__ void k_adj_dS(int p, const int* __restrict__ rowptr, const int* __restrict__ col,
                         const double* __restrict__ om, const double* __restrict__ x,
                         double* __restrict__ out, int ldo) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < p; i += nw) {
    double* orow = out + (size_t)i * ldo;
    for (int j = lane; j < p; j += 32) orow[j] = 0.0;
    __syncwarp();
    for (int tk = rowptr[i]; tk < rowptr[i + 1]; ++tk) {
      const int k = col[tk];
      const double w = om[tk];
      for (int t = rowptr[k] + lane; t < rowptr[k + 1]; t += 32) orow[col[t]] -= w * x[t];
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------- dL/dX
// Sparse products with the symmetric CSR matrices Omega (om) and Ahat (x):
// for R rows r of the dense n x p inputs, O[r, j] = sum_{t in row j}
// In[r, col[t]] * v[t].  The R input rows are staged in shared memory when
// they fit (STAGED), else read through L1.
//   split: P = Z Omega, Q = Z Ahat
//   merge: dZ = scale (P Ahat + Q Omega)
template <int R, bool STAGED>
__global__ void k_adj_spmm_split(const double* __restrict__ Z, int ldz, int n, int p,
                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ om, const double* __restrict__ ah,
                                 double* __restrict__ P, double* __restrict__ Q) {
  extern __shared__ double sm[];
  const int r0 = blockIdx.x * R;
  const int rows = min(R, n - r0);
  const double* in;
  int ldi;
  if (STAGED) {
    for (int rr = 0; rr < rows; ++rr)
      for (int c = threadIdx.x; c < p; c += blockDim.x) sm[rr * p + c] = Z[(size_t)(r0 + rr) * ldz + c];
    __syncthreads();
    in = sm;
    ldi = p;
  } else {
    in = Z + (size_t)r0 * ldz;
    ldi = ldz;
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    double ap[R], aq[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) ap[rr] = aq[rr] = 0.0;
    for (int t = rowptr[j]; t < rowptr[j + 1]; ++t) {
      const int c = col[t];
      const double wo = om[t], wa = ah[t];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        if (rr < rows) {
          const double zv = in[rr * ldi + c];
          ap[rr] = fma(zv, wo, ap[rr]);
          aq[rr] = fma(zv, wa, aq[rr]);
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      if (rr < rows) {
        P[(size_t)(r0 + rr) * ldz + j] = ap[rr];
        Q[(size_t)(r0 + rr) * ldz + j] = aq[rr];
      }
    }
  }
}

template <int R, bool STAGED>
__global__ void k_adj_spmm_merge(const double* __restrict__ P, const double* __restrict__ Q, int ldz,
                                 int n, int p, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, const double* __restrict__ om,
                                 const double* __restrict__ ah, double scale,
                                 double* __restrict__ dZ) {
  extern __shared__ double sm[];
  const int r0 = blockIdx.x * R;
  const int rows = min(R, n - r0);
  const double *ip, *iq;
  int ldi;
  if (STAGED) {
    for (int rr = 0; rr < rows; ++rr)
      for (int c = threadIdx.x; c < p; c += blockDim.x) {
        sm[rr * p + c] = P[(size_t)(r0 + rr) * ldz + c];
        sm[(R + rr) * p + c] = Q[(size_t)(r0 + rr) * ldz + c];
      }
    __syncthreads();
    ip = sm;
    iq = sm + (size_t)R * p;
    ldi = p;
  } else {
    ip = P + (size_t)r0 * ldz;
    iq = Q + (size_t)r0 * ldz;
    ldi = ldz;
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    double acc[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) acc[rr] = 0.0;
    for (int t = rowptr[j]; t < rowptr[j + 1]; ++t) {
      const int c = col[t];
      const double wo = om[t], wa = ah[t];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        if (rr < rows) acc[rr] = fma(ip[rr * ldi + c], wa, fma(iq[rr * ldi + c], wo, acc[rr]));
      }
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr < rows) dZ[(size_t)(r0 + rr) * ldz + j] = scale * acc[rr];
  }
}

// Column sums of dZ and dZ * Z over a chunk of rows: part1/part2[chunk * p + c].
__global__ void k_adj_colsum(const double* __restrict__ dZ, const double* __restrict__ Z, int ldz,
                             int n, int p, int rows_per_chunk, double* __restrict__ part1,
                             double* __restrict__ part2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(n, r0 + rows_per_chunk);
  double s1 = 0.0, s2 = 0.0;
  for (int r = r0; r < r1; ++r) {
    const double d = dZ[(size_t)r * ldz + c];
    s1 += d;
    s2 = fma(d, Z[(size_t)r * ldz + c], s2);
  }
  part1[(size_t)blockIdx.y * p + c] = s1;
  part2[(size_t)blockIdx.y * p + c] = s2;
}

__global__ void k_adj_colfin(const double* __restrict__ part1, const double* __restrict__ part2,
                             int chunks, int p, int n, double* __restrict__ m1,
                             double* __restrict__ m2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < chunks; ++k) {
    s1 += part1[(size_t)k * p + c];
    s2 += part2[(size_t)k * p + c];
  }
  m1[c] = s1 / n;
  m2[c] = s2 / n;
}

// Chain rule of Z = (X - mean) * s (prep 0: mean 0, s 1; prep 1: s 1):
//   dX = s (dZ - [prep >= 1] mean_r dZ - [prep == 2] Z mean_r(dZ Z)).
template <typename OutT>
__global__ void k_adj_dX(const double* __restrict__ dZ, const double* __restrict__ Z, int ldz, int n,
                         int p, int prep, const double* __restrict__ m1, const double* __restrict__ m2,
                         const double* __restrict__ inv_scale, OutT* __restrict__ dX, int lddx) {
  const size_t total = (size_t)n * p;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(k / p), c = (int)(k % p);
    double d = dZ[(size_t)r * ldz + c];
    if (prep >= 1) d -= m1[c];
    if (prep == 2) d = (d - Z[(size_t)r * ldz + c] * m2[c]) * inv_scale[c];
    dX[(size_t)r * lddx + c] = (OutT)d;
  }
}

inline int grid_for(size_t work, int block, int sms) {
  size_t g = (work + block - 1) / block;
  const size_t cap = (size_t)sms * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_adj_count(const void* Om, int f32, int p, int ld, int* cnt, int sms,
                             cudaStream_t st) {
  const int g = grid_for((size_t)p * 32, 256, sms);
  note_launches(1);
  if (f32) k_adj_count<float><<<g, 256, 0, st>>>((const float*)Om, p, ld, cnt);
  else k_adj_count<double><<<g, 256, 0, st>>>((const double*)Om, p, ld, cnt);
  return cudaGetLastError();
}

cudaError_t launch_adj_scan(const int* cnt, int p, int* rowptr, cudaStream_t st) {
  note_launches(1);
  k_adj_scan<<<1, 1024, 0, st>>>(cnt, p, rowptr);
  return cudaGetLastError();
}

cudaError_t launch_adj_fill(const void* Om, int f32, int p, int ld, const int* rowptr, int* col,
                            int* erow, double* om, int sms, cudaStream_t st) {
  const int g = grid_for((size_t)p * 32, 256, sms);
  note_launches(1);
  if (f32) k_adj_fill<float><<<g, 256, 0, st>>>((const float*)Om, p, ld, rowptr, col, erow, om);
  else k_adj_fill<double><<<g, 256, 0, st>>>((const double*)Om, p, ld, rowptr, col, erow, om);
  return cudaGetLastError();
}

cudaError_t launch_adj_prep(int nnz, const int* rowptr, const int* col, const int* erow,
                            const double* om, const double* sdiag, int* mirror, double* minv,
                            int* bad, int sms, cudaStream_t st) {
  note_launches(1);
  k_adj_prep<<<grid_for(nnz, 256, sms), 256, 0, st>>>(nnz, rowptr, col, erow, om, sdiag, mirror,
                                                      minv, bad);
  return cudaGetLastError();
}

cudaError_t launch_adj_rhs_dense(const void* g, int f32, int ldg, int nnz, const int* col,
                                 const int* erow, double* b, int sms, cudaStream_t st) {
  note_launches(1);
  const int gr = grid_for(nnz, 256, sms);
  if (f32) k_adj_rhs_dense<float><<<gr, 256, 0, st>>>((const float*)g, ldg, nnz, col, erow, b);
  else k_adj_rhs_dense<double><<<gr, 256, 0, st>>>((const double*)g, ldg, nnz, col, erow, b);
  return cudaGetLastError();
}

cudaError_t launch_adj_heldout(int nnz, const int* rowptr, const int* col, const int* erow,
                               const int* mirror, const double* om, const void* Sv, int sv_f32,
                               int lds, double* b, double* part, int part_cap, double* loss,
                               int sms, cudaStream_t st) {
  int g = grid_for((size_t)nnz * 32, 256, sms);
  if (g > part_cap) g = part_cap;
  note_launches(2);
  if (sv_f32)
    k_adj_heldout<float><<<g, 256, 0, st>>>(nnz, rowptr, col, erow, mirror, om, (const float*)Sv,
                                            lds, b, part);
  else
    k_adj_heldout<double><<<g, 256, 0, st>>>(nnz, rowptr, col, erow, mirror, om, (const double*)Sv,
                                             lds, b, part);
  k_adj_sum<<<1, 32, 0, st>>>(part, g, loss);
  return cudaGetLastError();
}

cudaError_t adj_cg_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_adj_cg, kAdjThreads, 0);
}

cudaError_t launch_adj_cg(const AdjArgs& a, int grid, cudaStream_t st) {
  note_launches(1);
  void* kargs[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)k_adj_cg, dim3(grid), dim3(kAdjThreads), kargs, 0,
                                     st);
}

cudaError_t launch_adj_dS(int p, const int* rowptr, const int* col, const double* om,
                          const double* x, double* out, int ldo, int sms, cudaStream_t st) {
  note_launches(1);
  k_adj_dS<<<grid_for((size_t)p * 32, 256, sms), 256, 0, st>>>(p, rowptr, col, om, x, out, ldo);
  return cudaGetLastError();
}

namespace {
constexpr size_t kSpmmSmem = 200 * 1024;

template <int R, bool STAGED>
cudaError_t spmm_pair(const double* Z, double* P, double* Q, double* dZ, int ldz, int n, int p,
                      const int* rowptr, const int* col, const double* om, const double* ah,
                      double scale, cudaStream_t st) {
  const int grid = (n + R - 1) / R;
  const size_t s1 = STAGED ? sizeof(double) * R * (size_t)p : 0;
  const size_t s2 = 2 * s1;
  cudaError_t e;
  if (STAGED) {
    e = cudaFuncSetAttribute(k_adj_spmm_split<R, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_adj_spmm_merge<R, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s2);
    if (e != cudaSuccess) return e;
  }
  note_launches(2);
  k_adj_spmm_split<R, STAGED><<<grid, 256, s1, st>>>(Z, ldz, n, p, rowptr, col, om, ah, P, Q);
  k_adj_spmm_merge<R, STAGED><<<grid, 256, s2, st>>>(P, Q, ldz, n, p, rowptr, col, om, ah, scale, dZ);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adj_data(const double* Z, double* P, double* Q, double* dZ, int ldz, int n, int p,
                            int prep, const int* rowptr, const int* col, const double* om,
                            const double* ah, const double* inv_scale, double* part1, double* part2,
                            double* m1, double* m2, void* dX, int dx_f32, int lddx, int sms,
                            cudaStream_t st) {
  const double scale = -1.0 / n;
  cudaError_t e;
  if (2 * sizeof(double) * 4 * (size_t)p <= kSpmmSmem)
    e = spmm_pair<4, true>(Z, P, Q, dZ, ldz, n, p, rowptr, col, om, ah, scale, st);
  else if (2 * sizeof(double) * (size_t)p <= kSpmmSmem)
    e = spmm_pair<1, true>(Z, P, Q, dZ, ldz, n, p, rowptr, col, om, ah, scale, st);
  else
    e = spmm_pair<4, false>(Z, P, Q, dZ, ldz, n, p, rowptr, col, om, ah, scale, st);
  if (e != cudaSuccess) return e;
  const int chunks = kAdjColChunks;
  const int rpc = (n + chunks - 1) / chunks;
  note_launches(prep >= 1 ? 3 : 1);
  if (prep >= 1) {
    k_adj_colsum<<<dim3((p + 255) / 256, chunks), 256, 0, st>>>(dZ, Z, ldz, n, p, rpc, part1, part2);
    k_adj_colfin<<<(p + 255) / 256, 256, 0, st>>>(part1, part2, chunks, p, n, m1, m2);
  }
  const int g = grid_for((size_t)n * p, 256, sms);
  if (dx_f32)
    k_adj_dX<float><<<g, 256, 0, st>>>(dZ, Z, ldz, n, p, prep, m1, m2, inv_scale, (float*)dX, lddx);
  else
    k_adj_dX<double><<<g, 256, 0, st>>>(dZ, Z, ldz, n, p, prep, m1, m2, inv_scale, (double*)dX, lddx);
  return cudaGetLastError();
}

}  // namespace concord
