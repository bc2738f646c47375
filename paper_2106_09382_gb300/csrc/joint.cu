// Joint two-population CONCORD: block coordinate descent on the joint
// objective that closes Section 6 (two precision matrices, lasso weight
// lambda1 on each, fusion weight lambda2 on |omega1_ij - omega2_ij| for
// i <= j), in S units.
//
// Layout on the GPU (one persistent cooperative launch runs whole sweeps):
//   * Colour steps follow Algorithm 1's circle-method schedule (closed form).
//     The blocks (omega1_ij, omega2_ij) of one colour touch disjoint rows, so
//     they are independent (the argument of Lemma 1 applies to the pair of
//     matrices unchanged): one grid barrier per colour step is the only
//     synchronisation.
//   * A colour's pairs are handed out one per warp (kJointWarps per CTA per
//     round).  The warp's lanes load the ten scalars of the pair at once
//     (W1_ij, W1_ji, W2_ij, W2_ji, the two old values, four diagonal S
//     entries); every lane solves the two-variable block problem in FP64.
//   * A pair that moved updates four W rows (W_m row i += d_m S_m row j,
//     row j += d_m S_m row i).  The whole CTA applies them with 16-byte
//     vectors: one warp alone keeps too few bytes in flight for a p-long row.
//   * After the last colour, the diagonal blocks (omega1_ii, omega2_ii), one
//     warp per row; then a fused pass over 32 x 32 tiles of the upper
//     triangle computes the joint KKT residual and the joint objective.
#include <math.h>

#include "joint.h"
#include "kernels.h"

namespace concord {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct JVec;
template <>
struct JVec<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static void fma(V& w, float d, const V& s) {
    w.x = fmaf(d, s.x, w.x);
    w.y = fmaf(d, s.y, w.y);
    w.z = fmaf(d, s.z, w.z);
    w.w = fmaf(d, s.w, w.w);
  }
};
template <>
struct JVec<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void fma(V& w, double d, const V& s) {
    w.x = ::fma(d, s.x, w.x);
    w.y = ::fma(d, s.y, w.y);
  }
};

// The block arithmetic runs in the working precision T: FP32 for the FP32
// sweeps (whose result the FP64 polish refines), FP64 for the FP64 sweeps.
// FP64 issues at a small fraction of the FP32 rate on this part and every
// colour step waits for its slowest block, so the block minimiser divides
// only in the branch it takes: the sign test x > y of the separated
// solutions is made on the numerators, cross-multiplied by the (positive)
// denominators.

template <typename T>
__device__ __forceinline__ T jsoft(T x, T tau) {
  const T a = fabs(x) - tau;
  if (!(a > (T)0)) return (T)0;
  return x > (T)0 ? a : -a;
}

// Minimiser of the block problem
//   c1 x^2 / 2 + g1 x + c2 y^2 / 2 + g2 y + l1 (|x| + |y|) + l2 |x - y|.
// With the sign of x - y fixed, the problem separates into two lasso
// problems whose solutions are the minimiser when they agree with that sign;
// if neither sign is consistent, the minimiser lies on x = y.
template <typename T>
__device__ __forceinline__ void block_pair(T c1, T g1, T c2, T g2, T l1, T l2, T& x, T& y) {
  const T na = jsoft<T>(-(g1 + l2), l1), nb = jsoft<T>(-(g2 - l2), l1);
  if (na * c2 > nb * c1) {  // na / c1 > nb / c2
    x = na / c1;
    y = nb / c2;
    return;
  }
  const T nc = jsoft<T>(-(g1 - l2), l1), nd = jsoft<T>(-(g2 + l2), l1);
  if (nc * c2 < nd * c1) {  // nc / c1 < nd / c2
    x = nc / c1;
    y = nd / c2;
    return;
  }
  const T nt = jsoft<T>(-(g1 + g2), (T)2 * l1);
  x = y = (nt == (T)0) ? (T)0 : nt / (c1 + c2);
}

// Positive root of s d^2 + b d - 1 = 0 (the stationarity condition of Eq. 2).
template <typename T>
__device__ __forceinline__ T pos_root(T s, T b) {
  return (-b + sqrt(b * b + (T)4 * s)) / ((T)2 * s);
}

// Minimiser over d1, d2 > 0 of
//   -log d1 + s1 d1^2 / 2 + b1 d1 - log d2 + s2 d2^2 / 2 + b2 d2 + l2 |d1 - d2|
// by the same three cases; the fused root solves (s1 + s2) d^2 + (b1 + b2) d = 2.
template <typename T>
__device__ __forceinline__ void block_diag(T s1, T b1, T s2, T b2, T l2, T& d1, T& d2) {
  const T ua = pos_root<T>(s1, b1 + l2), va = pos_root<T>(s2, b2 - l2);
  if (ua > va) {
    d1 = ua;
    d2 = va;
    return;
  }
  const T ub = pos_root<T>(s1, b1 - l2), vb = pos_root<T>(s2, b2 + l2);
  if (ub < vb) {
    d1 = ub;
    d2 = vb;
    return;
  }
  const T ss = s1 + s2, bb = b1 + b2;
  d1 = d2 = (-bb + sqrt(bb * bb + (T)8 * ss)) / ((T)2 * ss);
}

// max that propagates NaN (fmax would drop it).
template <typename T>
__device__ __forceinline__ T nmax(T a, T b) { return (a != a || a > b) ? a : b; }

template <typename T>
__device__ __forceinline__ T clampt(T v, T l) { return fmin(fmax(v, -l), l); }

template <typename T>
__device__ __forceinline__ T lasso_res(T g, T x, T l1) {
  if (x > (T)0) return fabs(g + l1);
  if (x < (T)0) return fabs(g - l1);
  return fmax(fabs(g) - l1, (T)0);
}

// Joint KKT residual of one pair block (smooth gradients g1, g2): the
// smallest, over the admissible fusion subgradient u = l2 z, of the larger of
// the two lasso residuals.  For x = y the larger residual is convex in u and
// smallest at the midpoint of the two gradients, clamped to [-l2, l2].
template <typename T>
__device__ __forceinline__ T pair_kkt(T g1, T g2, T x, T y, T l1, T l2) {
  if (x != y) {
    const T u = x > y ? l2 : -l2;
    return nmax<T>(lasso_res<T>(g1 + u, x, l1), lasso_res<T>(g2 - u, y, l1));
  }
  if (x != (T)0) {
    const T sg = x > (T)0 ? l1 : -l1;
    const T A = g1 + sg, B = g2 + sg;
    const T u = clampt<T>((T)0.5 * (B - A), l2);
    return nmax<T>(fabs(A + u), fabs(B - u));
  }
  const T u = clampt<T>((T)0.5 * (g2 - g1), l2);
  const T m = nmax<T>(fabs(g1 + u), fabs(g2 - u)) - l1;
  return m != m ? m : fmax(m, (T)0);
}

// Diagonal block: a = W1_ii - 1/d1, b = W2_ii - 1/d2, no lasso term.
template <typename T>
__device__ __forceinline__ T diag_kkt(T a, T b, T d1, T d2, T l2) {
  const T u = (d1 != d2) ? (d1 > d2 ? l2 : -l2) : clampt<T>((T)0.5 * (b - a), l2);
  return nmax<T>(fabs(a + u), fabs(b - u));
}

// The pair of slot q of colour c (Algorithm 1's rotation in closed form):
// vertex 0 stays put and meets the vertex at ring index P - 1; ring indices
// r and P - 2 - r face each other; during colour c the vertex at ring index r
// is ((r - c) mod P) + 1.  Returns (i, j) with i < j, or i = -1 for the bye
// of an odd p (the pair that holds vertex p); (ra, rb) are the slot's two
// vertices as they are (one of them is p for a bye).
__device__ __forceinline__ void slot_pair(int q, int c, int P, int p, int& i, int& j, int& ra,
                                          int& rb) {
  int a, b;
  if (q == 0) {
    a = 0;
    b = ((P - 1 - c) % P + P) % P + 1;
  } else {
    const int r = q - 1;
    a = ((r - c) % P + P) % P + 1;
    b = ((P - 2 - r - c) % P + P) % P + 1;
  }
  ra = a;
  rb = b;
  i = min(a, b);
  j = max(a, b);
  if (j >= p) i = -1;
}

// Row versions (dataflow between colour steps).  A row's version is the
// number of colour steps of this launch whose update of that row is complete
// and visible.  The pair of colour c of sweep t reads rows i and j only after
// both carry version t P + c; after its own update the CTA publishes
// t P + c + 1 for them (release after the CTA-wide barrier, so the writes of
// every thread of the CTA are covered).  Each vertex sits in exactly one slot
// of every colour (byes included), so every row is published every colour;
// waits only ever point to earlier colours, so the earliest CTA can always
// proceed.  Waits are bounded like every other wait of this library.
__device__ __forceinline__ void jst_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void wait_version(const unsigned* f, unsigned v, const WaitCtl& w,
                                             int row, int step) {
  if (ld_acquire_u32(f) >= v) return;
  const uint64_t t0 = globaltimer_ns();
  unsigned it = 0;
  while (ld_acquire_u32(f) < v) {
    if ((++it & 15u) == 0) {
      if (ld_relaxed_s32(w.abort) != 0) return;
      if (globaltimer_ns() - t0 > w.timeout_ns) {
        record_timeout(w, row, step);
        return;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void cta_axpy2(T* __restrict__ wi, T* __restrict__ wj,
                                          const T* __restrict__ si, const T* __restrict__ sj, T d,
                                          int ld) {
  using VT = JVec<T>;
  using V = typename VT::V;
  const int nv = ld / VT::N;
  V* wiv = reinterpret_cast<V*>(wi);
  V* wjv = reinterpret_cast<V*>(wj);
  const V* siv = reinterpret_cast<const V*>(si);
  const V* sjv = reinterpret_cast<const V*>(sj);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const V a = __ldg(sjv + v), b = __ldg(siv + v);
    V x = __ldcg(wiv + v), y = __ldcg(wjv + v);
    VT::fma(x, d, a);
    VT::fma(y, d, b);
    wiv[v] = x;
    wjv[v] = y;
  }
}

template <typename T>
__device__ __forceinline__ void warp_axpy(T* __restrict__ w, const T* __restrict__ s, T d, int ld,
                                          int lane) {
  using VT = JVec<T>;
  using V = typename VT::V;
  const int nv = ld / VT::N;
  V* wv = reinterpret_cast<V*>(w);
  const V* sv = reinterpret_cast<const V*>(s);
  for (int v = lane; v < nv; v += 32) {
    V x = wv[v];
    VT::fma(x, d, __ldg(sv + v));
    wv[v] = x;
  }
}

template <typename T>
__global__ void __launch_bounds__(kJointThreads, 1) k_joint(const JointArgs<T> a) {
  const int p = a.p, P = a.P, ld = a.ld;
  const int half = (P + 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double l1 = a.lambda1, l2 = a.lambda2;
  const T l1t = (T)l1, l2t = (T)l2;

  __shared__ int s_i[kJointWarps], s_j[kJointWarps];
  __shared__ T s_d[kJointWarps][2];
  __shared__ T wt[2][32][33];
  __shared__ double red[kJointWarps][kJParts];
  __shared__ double s_tot[kJParts];
  __shared__ int s_abort;

  unsigned gen = 0;
  int t = 0, first_delta = 0, evals = 0, since_best = 0;
  double best = INFINITY;
  int status = kJStatusMaxSweeps;
  double kkt = 0.0, obj = 0.0, delta = 0.0, moved_tot = 0.0;

  for (;;) {
    const bool initial = evals == 0 && a.eval_first;
    const bool swept = !initial && t < a.n_sweeps;
    T dmax = (T)0;  // lane-0 / thread-local contributions, kept in T (FP64 is slow here)
    int moved = 0;
    if (swept) {
      // ---- colour steps
      for (int c = 0; c < P; ++c) {
        for (int base = blockIdx.x * kJointWarps; base < half; base += gridDim.x * kJointWarps) {
          const int q = base + wid;
          int i = -1, j = -1, ra = p, rb = p;
          if (q < half) slot_pair(q, c, P, p, i, j, ra, rb);
          const unsigned vin = (unsigned)(t * P + c);
          // failure testing: the row that skips its publication at this step
          const int skip = (a.fault_step >= 0 && vin == (unsigned)a.fault_step) ? a.fault_row : -1;
          if (a.row_ver != nullptr && q < half) {
            const int r = lane == 0 ? ra : rb;
            if (lane < 2 && r < p) wait_version(a.row_ver + r, vin, a.wait, r, c);
            __syncwarp();
          }
          T d0 = (T)0, d1 = (T)0;
          if (i >= 0) {
            const size_t ij = (size_t)i * ld + j, ji = (size_t)j * ld + i;
            const size_t ii = (size_t)i * ld + i, jj = (size_t)j * ld + j;
            T v = (T)0;
            switch (lane) {
              case 0: v = __ldcg(a.W[0] + ij); break;
              case 1: v = __ldcg(a.W[0] + ji); break;
              case 2: v = __ldcg(a.W[1] + ij); break;
              case 3: v = __ldcg(a.W[1] + ji); break;
              case 4: v = __ldcg(a.Om[0] + ij); break;
              case 5: v = __ldcg(a.Om[1] + ij); break;
              case 6: v = __ldg(a.S[0] + ii); break;
              case 7: v = __ldg(a.S[0] + jj); break;
              case 8: v = __ldg(a.S[1] + ii); break;
              case 9: v = __ldg(a.S[1] + jj); break;
              default: break;
            }
            const T w1ij = __shfl_sync(kFull, v, 0), w1ji = __shfl_sync(kFull, v, 1);
            const T w2ij = __shfl_sync(kFull, v, 2), w2ji = __shfl_sync(kFull, v, 3);
            const T o1 = __shfl_sync(kFull, v, 4), o2 = __shfl_sync(kFull, v, 5);
            const T s1i = __shfl_sync(kFull, v, 6), s1j = __shfl_sync(kFull, v, 7);
            const T s2i = __shfl_sync(kFull, v, 8), s2j = __shfl_sync(kFull, v, 9);
            // smooth gradient without the pair's own quadratic term (the two
            // direct sums of Eq. 3): W_ij + W_ji - (s_ii + s_jj) w_ij
            const T c1 = s1i + s1j, c2 = s2i + s2j;
            const T g1 = (w1ij + w1ji) - c1 * o1;
            const T g2 = (w2ij + w2ji) - c2 * o2;
            T xn, yn;
            block_pair<T>(c1, g1, c2, g2, l1t, l2t, xn, yn);
            d0 = xn - o1;
            d1 = yn - o2;
            if (lane == 0) {
              if (d0 != (T)0) {
                a.Om[0][ij] = xn;
                a.Om[0][ji] = xn;
              }
              if (d1 != (T)0) {
                a.Om[1][ij] = yn;
                a.Om[1][ji] = yn;
              }
              dmax = nmax<T>(dmax, nmax<T>(fabs(d0), fabs(d1)));
              if (d0 != (T)0 || d1 != (T)0) ++moved;
            }
          }
          const bool mv = d0 != (T)0 || d1 != (T)0;  // the same on every lane
          if (lane == 0) {
            s_i[wid] = i;
            s_j[wid] = j;
            s_d[wid][0] = d0;
            s_d[wid][1] = d1;
          }
          // A block that did not move (or a bye) left its rows untouched and
          // its reads are complete: publish them now, so the readers of the
          // next colour do not wait for this CTA's row updates.
          if (a.row_ver != nullptr && lane == 0 && q < half && !mv) {
            if (ra < p && ra != skip) jst_release_u32(a.row_ver + ra, vin + 1u);
            if (rb < p && rb != skip) jst_release_u32(a.row_ver + rb, vin + 1u);
          }
          if (__syncthreads_or(lane == 0 && mv)) {
            for (int w = 0; w < kJointWarps; ++w) {
              const int i2 = s_i[w];
              if (i2 < 0) continue;
              const int j2 = s_j[w];
#pragma unroll
              for (int m = 0; m < 2; ++m) {
                const T d = s_d[w][m];
                if (d == (T)0) continue;
                cta_axpy2<T>(a.W[m] + (size_t)i2 * ld, a.W[m] + (size_t)j2 * ld,
                             a.S[m] + (size_t)i2 * ld, a.S[m] + (size_t)j2 * ld, d, ld);
              }
            }
            __syncthreads();
            if (a.row_ver != nullptr && lane == 0 && q < half && mv) {
              if (ra < p && ra != skip) jst_release_u32(a.row_ver + ra, vin + 1u);
              if (rb < p && rb != skip) jst_release_u32(a.row_ver + rb, vin + 1u);
            }
          }
        }
        if (a.row_ver == nullptr) grid_barrier(a.barrier, gen, a.wait, c);
      }
      if (a.row_ver != nullptr) grid_barrier(a.barrier, gen, a.wait, P - 1);
      // ---- diagonal blocks, one warp per row
      const int tw = gridDim.x * kJointWarps;
      for (int i = blockIdx.x * kJointWarps + wid; i < p; i += tw) {
        const size_t ii = (size_t)i * ld + i;
        T v = (T)0;
        switch (lane) {
          case 0: v = a.W[0][ii]; break;
          case 1: v = a.W[1][ii]; break;
          case 2: v = a.Om[0][ii]; break;
          case 3: v = a.Om[1][ii]; break;
          case 4: v = __ldg(a.S[0] + ii); break;
          case 5: v = __ldg(a.S[1] + ii); break;
          default: break;
        }
        const T w1 = __shfl_sync(kFull, v, 0), w2 = __shfl_sync(kFull, v, 1);
        const T o1 = __shfl_sync(kFull, v, 2), o2 = __shfl_sync(kFull, v, 3);
        const T s1 = __shfl_sync(kFull, v, 4), s2 = __shfl_sync(kFull, v, 5);
        // the direct sum of Eq. 2: W_ii - w_ii s_ii
        const T b1 = w1 - o1 * s1;
        const T b2 = w2 - o2 * s2;
        T n1, n2;
        block_diag<T>(s1, b1, s2, b2, l2t, n1, n2);
        const T d0 = n1 - o1, d1 = n2 - o2;
        if (lane == 0) {
          if (d0 != (T)0) a.Om[0][ii] = n1;
          if (d1 != (T)0) a.Om[1][ii] = n2;
          dmax = nmax<T>(dmax, nmax<T>(fabs(d0), fabs(d1)));
        }
        if (d0 != (T)0) warp_axpy<T>(a.W[0] + (size_t)i * ld, a.S[0] + (size_t)i * ld, d0, ld, lane);
        if (d1 != (T)0) warp_axpy<T>(a.W[1] + (size_t)i * ld, a.S[1] + (size_t)i * ld, d1, ld, lane);
      }
      grid_barrier(a.barrier, gen, a.wait, P);
    }

    // ---- fused KKT / objective pass over the upper-triangle tiles
    // per-thread partials in T (a few dozen terms each), combined in FP64
    T kk = (T)0, quad = (T)0, logs = (T)0, pen = (T)0, fuse = (T)0;
    const int nt = (p + 31) / 32;
    for (int k = blockIdx.x; k < nt * nt; k += gridDim.x) {
      const int bi = k / nt, bj = k % nt;
      if (bi > bj) continue;
      // wt[m][c][r] = W_m[32 bj + r][32 bi + c]
      for (int e = threadIdx.x; e < 2 * 1024; e += blockDim.x) {
        const int m = e >> 10, r = (e >> 5) & 31, c = e & 31;
        const int row = 32 * bj + r;
        wt[m][c][r] = row < p ? a.W[m][(size_t)row * ld + 32 * bi + c] : (T)0;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        const int ty = e >> 5, tx = e & 31;
        const int i = 32 * bi + ty, j = 32 * bj + tx;
        if (i >= p || j >= p || i > j) continue;
        const size_t ij = (size_t)i * ld + j;
        const T x = a.Om[0][ij], y = a.Om[1][ij];
        const T wa = a.W[0][ij], wb = a.W[1][ij];
        if (i == j) {
          const T ga = wa - (T)1 / x, gb = wb - (T)1 / y;
          kk = nmax<T>(kk, diag_kkt<T>(ga, gb, x, y, l2t));
          quad += x * wa + y * wb;
          logs += log(x) + log(y);
          fuse += fabs(x - y);
        } else {
          const T g1 = wa + wt[0][ty][tx], g2 = wb + wt[1][ty][tx];
          kk = nmax<T>(kk, pair_kkt<T>(g1, g2, x, y, l1t, l2t));
          quad += x * g1 + y * g2;
          pen += fabs(x) + fabs(y);
          fuse += fabs(x - y);
        }
      }
      __syncthreads();
    }
    // block reduction of the partials
    {
      double v[kJParts] = {(double)kk, (double)quad, (double)logs, (double)pen, (double)fuse,
                           (double)dmax, (double)moved, 0.0};
#pragma unroll
      for (int q = 0; q < kJParts; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_down_sync(kFull, x, o);
          x = (q == kJPartKkt || q == kJPartDelta) ? nmax<double>(x, y) : x + y;
        }
        if (lane == 0) red[wid][q] = x;
      }
      __syncthreads();
      if (threadIdx.x < kJParts) {
        const int q = threadIdx.x;
        double x = red[0][q];
        for (int w = 1; w < kJointWarps; ++w)
          x = (q == kJPartKkt || q == kJPartDelta) ? nmax<double>(x, red[w][q]) : x + red[w][q];
        a.partials[((size_t)(evals & 1) * gridDim.x + blockIdx.x) * kJParts + q] = x;
      }
    }
    grid_barrier(a.barrier, gen, a.wait, P + 1);
    // every CTA combines the partials in the same order: the same decision
    if (wid == 0) {
      const double* part = a.partials + (size_t)(evals & 1) * gridDim.x * kJParts;
#pragma unroll 1
      for (int q = 0; q < kJParts; ++q) {
        const bool mx = (q == kJPartKkt || q == kJPartDelta);
        double x = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) {
          const double y = part[(size_t)b * kJParts + q];
          x = mx ? nmax<double>(x, y) : x + y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(kFull, x, o);
          x = mx ? nmax<double>(x, y) : x + y;
        }
        if (lane == 0) s_tot[q] = x;
      }
      if (lane == 0) s_abort = ld_relaxed_s32(a.wait.abort);
    }
    __syncthreads();
    ++evals;
    kkt = s_tot[kJPartKkt];
    obj = -s_tot[kJPartLog] + 0.5 * s_tot[kJPartQuad] + l1 * s_tot[kJPartPen] +
          l2 * s_tot[kJPartFuse];
    const bool finite = isfinite(kkt) && isfinite(obj);
    if (swept) {
      delta = s_tot[kJPartDelta];
      moved_tot = s_tot[kJPartMoved];
      if (blockIdx.x == 0 && threadIdx.x == 0 && t < a.hist_len) {
        double* h = a.hist + (size_t)t * kJHist;
        h[0] = delta;
        h[1] = kkt;
        h[2] = obj;
        h[3] = moved_tot;
      }
      ++t;
      if (!first_delta && delta < a.delta_tol) first_delta = t;
      if (kkt < 0.9 * best) {
        best = kkt;
        since_best = 0;
      } else {
        ++since_best;
      }
    }
    if (s_abort) {
      status = kJStatusAborted;
      break;
    }
    if (!finite) {
      status = kJStatusNonfinite;
      break;
    }
    if (kkt <= a.tol) {
      status = kJStatusConverged;
      break;
    }
    if (swept && a.stall_stop && since_best >= kJStallSweeps) {
      status = kJStatusStalled;
      break;
    }
    if (t >= a.n_sweeps) {
      status = kJStatusMaxSweeps;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.result[kJResSweeps] = t;
    a.result[kJResKkt] = kkt;
    a.result[kJResObj] = obj;
    a.result[kJResDelta] = delta;
    a.result[kJResMoved] = moved_tot;
    a.result[kJResStatus] = status;
    a.result[kJResFirstDelta] = first_delta;
  }
}

// W = Om S from the nonzero entries of each row of Om: one warp per row; the
// row's nonzeros are gathered by ballot in batches of 32 and applied to the
// whole W row (FP64 accumulation within a batch).
template <typename T>
__global__ void __launch_bounds__(256) k_joint_refresh(const T* __restrict__ Om,
                                                       const T* __restrict__ S, T* __restrict__ W,
                                                       int p, int ld) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= p) return;
  const T* o = Om + (size_t)row * ld;
  T* w = W + (size_t)row * ld;
  for (int c = lane; c < ld; c += 32) w[c] = (T)0;
  __syncwarp();
  for (int k0 = 0; k0 < p; k0 += 32) {
    const int k = k0 + lane;
    const T v = k < p ? o[k] : (T)0;
    unsigned nz = __ballot_sync(kFull, v != (T)0);
    if (!nz) continue;
    for (int c = lane; c < ld; c += 32) {
      double acc = (double)w[c];
      unsigned m = nz;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const double ov = (double)__shfl_sync(kFull, v, b);
        acc += ov * (double)__ldg(S + (size_t)(k0 + b) * ld + c);
      }
      w[c] = (T)acc;
    }
    __syncwarp();
  }
}

template <typename T>
cudaError_t launch_joint_t(const JointArgs<T>& a, int grid, cudaStream_t st) {
  if (a.ld % 32 != 0 || a.p < 2 || grid < 1) return cudaErrorInvalidValue;
  void* args[] = {(void*)&a};
  note_launches(1);
  return cudaLaunchCooperativeKernel((const void*)k_joint<T>, dim3(grid), dim3(kJointThreads),
                                     args, 0, st);
}

}  // namespace

cudaError_t launch_joint(const JointArgs<double>& a, int grid, cudaStream_t st) {
  return launch_joint_t(a, grid, st);
}
cudaError_t launch_joint(const JointArgs<float>& a, int grid, cudaStream_t st) {
  return launch_joint_t(a, grid, st);
}

cudaError_t joint_occupancy(bool f32, int* blocks_per_sm) {
  return f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_joint<float>,
                                                             kJointThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_joint<double>,
                                                             kJointThreads, 0);
}

cudaError_t launch_joint_refresh(const void* Om, const void* S, void* W, int p, int ld, bool f32,
                                 cudaStream_t st) {
  if (p < 1 || ld % 32 != 0) return cudaErrorInvalidValue;
  const int rows_per_block = 8;
  const int grid = (p + rows_per_block - 1) / rows_per_block;
  note_launches(1);
  if (f32)
    k_joint_refresh<float><<<grid, 256, 0, st>>>((const float*)Om, (const float*)S, (float*)W, p,
                                                 ld);
  else
    k_joint_refresh<double><<<grid, 256, 0, st>>>((const double*)Om, (const double*)S, (double*)W,
                                                  p, ld);
  return cudaGetLastError();
}

}  // namespace concord
