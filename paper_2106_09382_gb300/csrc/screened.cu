// Screened CONCORD-PCD sweep: the same iterates as Algorithm 1, computed by
// visiting only the pairs that can change.
//
// Why: in a colour step a pair (i, j) reads W_ij and W_ji as they stand after
// every earlier change of rows i and j in the sweep (Eq. 3 in W form), and
// nothing else (Lemma 1).  A pair whose soft-threshold stays at zero from
// w_ij = 0 changes nothing, so it can be skipped without affecting any other
// pair.  Near a solution only the support (a few per row) changes; the
// remaining ~p^2/2 pairs are zero and stay zero.  The colour loop then turns
// into a short dependency chain through the changed pairs, which one thread
// walks at register speed instead of the whole grid paying one exchange
// latency per colour step.
//
// One sweep (all CTAs, grid barriers between phases):
//   screen   every pair with w_ij != 0 or |W_ij + W_ji| > lambda at the sweep
//            start is a candidate (fused into the previous sweep's KKT pass);
//   build    candidates sorted by the colour step that visits them
//            (closed form of the circle method), per-row candidate lists in
//            step order, and for each candidate the S entries that carry the
//            earlier changes of its two rows into W_ij and W_ji;
//   chain    one thread evaluates Eq. 3 for the candidates in step order:
//            W_ij = W_ij(start) + sum over earlier changes (i, u, d) of d S_uj
//            (the lazily applied row updates, in step order);
//   rows     per row: W after the colour steps, the diagonal root (Eq. 2),
//            W += dw S_i, and V_ij = W_ij at the step that visits (i, j);
//   verify   every non-candidate pair must satisfy |V_ij + V_ji| <= lambda,
//            i.e. Eq. 3 leaves it at zero given the candidates' changes.  If
//            one does not, the sweep is undone, the failing pairs join the
//            candidates and the sweep is redone; the verification pass also
//            computes the objective and KKT residual and screens the next
//            sweep.
// The floating-point operations per pair are those of the dense sweep kernel
// (same FMA chains in the same order), so both kernels produce the same
// iterates.
#include "common.cuh"
#include "kernels.h"

namespace concord {

// How a sweep ends (see the decision in the kernel).
constexpr int kModeFull = 0, kModeLazy = 1, kModeDefer = 2, kModePartial = 3;

// Candidates of one row sorted by a warp in shared memory (longer rows: one
// thread, insertion sort).
constexpr int kSortCap = 512;
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float fma_t(float d, float s, float w) { return fmaf(d, s, w); }
__device__ __forceinline__ double fma_t(double d, double s, double w) { return ::fma(d, s, w); }

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static void split(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static V join(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void split(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static V join(const double* o) { return make_double2(o[0], o[1]); }
};

__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

__device__ __forceinline__ float nan_t(float) { return __int_as_float(0x7fffffff); }
__device__ __forceinline__ double nan_t(double) { return __longlong_as_double(0x7fffffffffffffffll); }

// High 32 bits of |v| as an unsigned integer: for finite values their order
// is the order of the magnitudes (IEEE layout), up to the low mantissa bits
// of doubles, which only makes the test below conservative.
__device__ __forceinline__ unsigned mag_hi(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ unsigned mag_hi(double v) {
  return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
}
// Largest high word whose magnitudes are all below `bound` (> 0).
__device__ __forceinline__ unsigned mag_hi_below(float bound) { return __float_as_uint(bound) - 1u; }
__device__ __forceinline__ unsigned mag_hi_below(double bound) {
  return (unsigned)((unsigned long long)__double_as_longlong(bound) >> 32) - 1u;
}


// Exclusive prefix sum by one CTA: out[k] = sum_{q<k} f(q) for k <= n (and
// the same into out2 when given).
template <typename F>
__device__ void cta_scan(F f, int n, int* out, int* out2, int* s_tmp, int* terms_out = nullptr) {
  const int nt = blockDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (n + nt - 1) / nt;
  const int b = min(n, threadIdx.x * per), e = min(n, b + per);
  int sum = 0;
  unsigned long long terms = 0ull;  // sum over the rows of c (c - 1) / 2
#pragma unroll 8
  for (int k = b; k < e; ++k) {  // independent loads: unrolled, in flight together
    const int c = f(k);
    sum += c;
    terms += (unsigned long long)c * (unsigned long long)(c > 0 ? c - 1 : 0) / 2ull;
  }
  if (terms_out != nullptr) {
    __shared__ unsigned long long s_terms_sum;
    if (threadIdx.x == 0) s_terms_sum = 0ull;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) terms += __shfl_down_sync(FULL, terms, o);
    if (lane == 0) atomicAdd(&s_terms_sum, terms);
    __syncthreads();
    if (threadIdx.x == 0)
      *terms_out = s_terms_sum > 0x7fffffffull ? 0x7fffffff : (int)s_terms_sum;
  }
  int x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int v = lane < (nt >> 5) ? s_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, v, o);
      if (lane >= o) v += y;
    }
    if (lane < (nt >> 5)) s_tmp[lane] = v;
  }
  __syncthreads();
  int run = x - sum + (wid > 0 ? s_tmp[wid - 1] : 0);
#pragma unroll 8
  for (int k = b; k < e; ++k) {
    const int c = f(k);
    out[k] = run;
    if (out2) out2[k] = run;
    run += c;
  }
  if (threadIdx.x == nt - 1) {
    out[n] = run;
    if (out2) out2[n] = run;
  }
  __syncthreads();
}

// Correction terms a list needs come with the scan (terms_out): a row with c
// candidates gives them 0 + 1 + ... + (c - 1) terms, saturated at INT_MAX, so
// a sweep whose terms cannot fit goes to the dense kernel before any is built.


template <typename T>
__device__ __forceinline__ void load8(const T* src, T (&o)[8]) {
  using VT = Vec<T>;
  using V = typename VT::V;
  const V* v = reinterpret_cast<const V*>(src);
#pragma unroll
  for (int q = 0; q < 8 / VT::N; ++q) VT::split(__ldcg(v + q), o + q * VT::N);
}

// Block reduction of the per-thread partials into partials[blockIdx.x*kParts+k].
__device__ __forceinline__ void reduce_parts(double (&v)[kParts], double* out,
                                             double (*red)[kParts]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < kParts; ++k) {
    double x = v[k];
    // most warps hold no terms of a part: skip their shuffle tree (tested on
    // the bits, with integer operations: the FP64 pipe is narrow on this
    // part, and 512 threads x 8 parts of FP64 compares and trees cost
    // microseconds per sweep).  The maxima are of nonnegative values, whose
    // bit patterns order as integers
    const long long xb = __double_as_longlong(x);
    if (__any_sync(FULL, (xb << 1) != 0ll)) {
      if (k == kPartKkt || k == kPartDelta) {
        long long m = xb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(FULL, m, o));
        x = __longlong_as_double(m);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
      }
    }
    if (lane == 0) red[wid][k] = x;
  }
  __syncthreads();
  // the warps' values, part by part, over the lanes of warp 0 (a fixed tree;
  // one thread adding them in turn was a chain of ~128 FP64 operations)
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < kParts; ++k) {
      double x = lane < nw ? red[lane][k] : 0.0;  // 0: the identity of both
      if (k == kPartKkt || k == kPartDelta) {
        long long m = __double_as_longlong(x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(FULL, m, o));
        x = __longlong_as_double(m);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
      }
      if (lane == 0) out[(size_t)blockIdx.x * kParts + k] = x;
    }
  }
  __syncthreads();
}

// Appends (i, j) for every lane whose predicate holds (all 32 lanes call).
__device__ __forceinline__ void push_list(bool pred, int i, int j, int2* list, int* count, int cap,
                                          int lane) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (pred) {
    const int r = base + __popc(m & ((1u << lane) - 1u));
    if (r < cap) list[r] = make_int2(i, j);
  }
}

// Appends (i, j) to a candidate list and counts it for both rows.
__device__ __forceinline__ void push_cand(bool pred, int i, int j, int2* list, int* count,
                                          int* cnt_r, int cap, int lane) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (pred) {
    const int r = base + __popc(m & ((1u << lane) - 1u));
    if (r < cap) {
      list[r] = make_int2(i, j);
      atomicAdd(cnt_r + i, 1);
      atomicAdd(cnt_r + j, 1);
    }
  }
}


// Screen of a launch's starting point over the upper triangle, in 8-row
// chunks of 32 x 32 tiles (lane l takes column j = tb*32 + l; W_ji comes from
// row j as one 8-element vector): (i, j) is a candidate when w_ij != 0 or
// |(0 - W_ij) - W_ji| > lambda.  With do_kkt it also forms the objective and
// KKT terms of the whole matrix (diagonal included).
template <typename T, bool MIXED>
__device__ void screen_pass(const ScreenArgs<T>& a, const T* __restrict__ W, int lst, bool do_kkt,
                            double lamd, double (&v)[kParts], int lane, int gwarp, int gwarps) {
  const int p = a.p, ld = a.ld;
  const ScreenWork<T>& w = a.w;
  const int nb = (p + kTile - 1) / kTile;
  const T lam_s = (T)(lamd * (1.0 - kScreenMargin));
  const int units = nb * nb * 4;
  for (int u = gwarp; u < units; u += gwarps) {
    const int tau = u >> 2, r0 = (u & 3) * 8;
    const int ta = tau / nb, tb = tau % nb;
    if (ta > tb) continue;
    const int j = tb * kTile + lane;
    const int i0 = ta * kTile + r0;
    if (i0 >= p) continue;
    const bool jv = j < p;
    T w1[8], om8[8], wt[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      const bool ok = jv && i < p;
      w1[r] = ok ? __ldcg(W + (size_t)i * ld + j) : (T)0;
      om8[r] = ok ? __ldcg(a.Om + (size_t)i * ld + j) : (T)0;
    }
    if (jv)
      load8(W + (size_t)j * ld + i0, wt);
    else
#pragma unroll
      for (int r = 0; r < 8; ++r) wt[r] = (T)0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      const bool pair = jv && i < p && i < j;
      const T x0 = ((T)0 - w1[r]) - wt[r];
      const bool cand = pair && (om8[r] != (T)0 || fabs(x0) - lam_s > (T)0);
      push_cand(cand, i, j, w.cand[lst], w.ctr + kCtrCand + lst, w.cnt_r[lst], w.nc_cap, lane);
    }
    if (!do_kkt) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      if (!jv || i >= p) continue;
      if (i < j) {
        const double om = (double)om8[r];
        const double g = (double)w1[r] + (double)wt[r];
        v[kPartKkt] = fmax(v[kPartKkt], kkt_offdiag(om, g, lamd));
        v[kPartQuad] += om * g;
        v[kPartPen] += fabs(om);
        if (!isfinite(g) || !isfinite(om)) v[kPartBad] += 1.0;
      } else if (i == j) {
        const double wii = (double)w1[r];
        const double oii = MIXED ? __ldcg(a.omdiag64 + i) : (double)om8[r];
        if (oii > 0.0 && isfinite(wii) && isfinite(oii)) {
          v[kPartKkt] = fmax(v[kPartKkt], fabs(wii - 1.0 / oii));
          v[kPartQuad] += oii * wii;
          v[kPartLog] += log(oii);
        } else {
          v[kPartBad] += 1.0;
        }
      }
    }
  }
}

// Deferred row updates (lazy sweeps).  Row i's true W_ix is its stored value
// with the row's pending (u, d) entries applied in order, w <- d S_ux + w:
// the FMA chain the dense kernel applies when the updates happen.
template <typename T>
__device__ __forceinline__ T pend_fold(const ScreenArgs<T>& a, int i, int n, int x, T wv) {
  const int* pu = a.w.pend_u + (size_t)i * kPendRow;
  const T* pd = a.w.pend_d + (size_t)i * kPendRow;
  for (int k0 = 0; k0 < n; k0 += 8) {  // loads in batches, then the FMAs in order
    int u[8];
    T d[8], sv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      u[r] = k0 + r < n ? ldi(pu + k0 + r) : -1;
      d[r] = k0 + r < n ? __ldcg(pd + k0 + r) : (T)0;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) sv[r] = u[r] >= 0 ? __ldg(a.S + (size_t)u[r] * a.ld + x) : (T)0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (u[r] >= 0) wv = fma_t(d[r], sv[r], wv);
  }
  return wv;
}

// Brings every stored row with pending entries up to date, in place: two work
// items per row (halves of its columns), each lane its own 16-byte vectors,
// the entries read by every lane (the same addresses: broadcast loads) and
// applied in order.  The caller zeroes the pending counts after a barrier
// (both halves read them here).
template <typename T>
__device__ void flush_pending(const ScreenArgs<T>& a, T* __restrict__ W, int lane, int gwarp,
                              int gwarps) {
  using VT = Vec<T>;
  using VV = typename VT::V;
  constexpr int VN = VT::N;
  const int p = a.p, ld = a.ld;
  const ScreenWork<T>& w = a.w;
  const int nv = ld / VN;
  for (int item = gwarp; item < 2 * p; item += gwarps) {
    const int i = item >> 1, half = item & 1;
    const int np = ldi(w.pend_n + i);
    if (np == 0) continue;
    const int qbeg = half ? nv / 2 : 0, qend = half ? nv : nv / 2;
    const int* pu = w.pend_u + (size_t)i * kPendRow;
    const T* pd = w.pend_d + (size_t)i * kPendRow;
    VV* row = reinterpret_cast<VV*>(W + (size_t)i * ld);
    for (int q = qbeg + lane; q < qend; q += 32) {
      T acc[VN];
      VT::split(__ldcg(row + q), acc);
      for (int k = 0; k < np; ++k) {
        const int u = ldi(pu + k);
        const T d = __ldcg(pd + k);
        T sv[VN];
        VT::split(__ldg(reinterpret_cast<const VV*>(a.S + (size_t)u * ld) + q), sv);
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[e] = fma_t(d, sv[e], acc[e]);
      }
      row[q] = VT::join(acc);
    }
  }
}

// After a sweep, over the pairs outside the candidates (V_ij not NaN; every
// such pair has w_ij = 0): the verification |(0 - V_ij) - V_ji| <= lambda
// (Eq. 3's test for staying at zero; a failing pair joins the fail list),
// their KKT terms max(|G_ij| - lambda, 0), and the screen of the next sweep.
// Only W and V are read; the candidates' own terms come from the candidate
// list and the diagonal's from the row pass.  Kept out of line: compiled
// inside the sweep kernel's body its loads were scheduled less well (the
// pass ran about 10% of a sweep slower).
// Partial verification (a sweep whose per-row bound fails only on a few
// "loud" rows): the pairs (i, j) of the loud rows i that are not candidates,
// with the same tests as verify_pass -- Eq. 3's zero test at the visit, the
// next sweep's screen and the KKT term after the sweep.  W_ij at the visit
// and after the sweep come from the stored row with its pending entries
// (the rows are not updated in such a sweep): the old entries, then the
// sweep's changes in step order (the visit value is taken before the first
// change at a later step), then the diagonal change -- the FMA order of a
// flush followed by the row pass, so the decisions are the full pass's.
// One warp per (loud row, 32 columns); a pair of two loud rows is taken by
// the smaller row.  Failing pairs go to the fail list, screened pairs to the
// next list's slot (merged into the kept list once the sweep stands).
template <typename T>
__device__ __forceinline__ void row_at_visit(const ScreenArgs<T>& a, const T* __restrict__ W, int r,
                                             int c, int c_step, T& at_visit, T& after) {
  const ScreenWork<T>& w = a.w;
  const int P = a.P, ld = a.ld;
  const int npo = ldi(w.pend_n + r), npn = ldi(w.pend_new + r);
  const int* pu = w.pend_u + (size_t)r * kPendRow;
  const T* pd = w.pend_d + (size_t)r * kPendRow;
  T acc = pend_fold(a, r, npo, c, __ldcg(W + (size_t)r * ld + c));
  T vis = acc;
  bool cap = false;
  for (int m0 = npo; m0 < npn; m0 += 8) {  // loads in batches, then the FMAs in order
    int u[8];
    T d[8], sv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      u[q] = m0 + q < npn ? ldi(pu + m0 + q) : -1;
      d[q] = m0 + q < npn ? __ldcg(pd + m0 + q) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sv[q] = u[q] >= 0 ? __ldg(a.S + (size_t)u[q] * ld + c) : (T)0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (u[q] < 0) break;
      // the diagonal change (u == r) follows every colour step
      const int cm = u[q] == r ? 0x7fffffff : pair_step(min(r, u[q]), max(r, u[q]), P);
      if (!cap && cm > c_step) {
        vis = acc;
        cap = true;
      }
      acc = fma_t(d[q], sv[q], acc);
    }
  }
  at_visit = cap ? vis : acc;
  after = acc;
}

template <typename T>
__device__ __noinline__ void partial_verify(const ScreenArgs<T>& a, const T* __restrict__ W, int cur,
                                            int nloud, double lamd, double (&v)[kParts], int lane,
                                            int swarp, int gwarps) {
  const int p = a.p, P = a.P;
  const ScreenWork<T>& w = a.w;
  const T lam = (T)lamd;
  const T lam_s = (T)(lamd * (1.0 - kScreenMargin));
  const int nchunk = (p + 31) >> 5;
  const int nxt = 1 - cur;
  for (int item = swarp; item < nloud * nchunk; item += gwarps) {
    const int i = ldi(w.loud + item / nchunk);
    const int j = (item % nchunk) * 32 + lane;
    bool pair = j < p && j != i;
    if (pair && j < i && ldi(w.loudf + j) != 0) pair = false;
    {  // candidates are not verified: the row's partners, 32 at a time
      const int b = ldi(w.off_r + i), ne = ldi(w.off_r + i + 1) - b;
      for (int m0 = 0; m0 < ne; m0 += 32) {
        int mine = -1;
        if (m0 + lane < ne) {
          const int2 qp = __ldcg(w.cand[cur] + ldi(w.row_ent + b + m0 + lane));
          mine = qp.x == i ? qp.y : qp.x;
        }
        const int nm = min(32, ne - m0);
        for (int m = 0; m < nm; ++m)
          if (__shfl_sync(FULL, mine, m) == j) pair = false;
      }
    }
    bool bad = false, next = false;
    if (pair) {
      const int c_step = pair_step(min(i, j), max(i, j), P);
      T vij, wij, vji, wji;
      row_at_visit(a, W, i, j, c_step, vij, wij);
      row_at_visit(a, W, j, i, c_step, vji, wji);
      bad = fabs(((T)0 - vij) - vji) - lam > (T)0;
      next = fabs(((T)0 - wij) - wji) - lam_s > (T)0;
      const double g = (double)wij + (double)wji;
      v[kPartKkt] = fmax(v[kPartKkt], fmax(fabs(g) - lamd, 0.0));
      if (!isfinite(g)) v[kPartBad] += 1.0;
    }
    const int lo = min(i, j), hi = max(i, j);
    push_list(bad, lo, hi, w.fail, w.ctr + kCtrFail, w.fail_cap, lane);
    push_cand(next, lo, hi, w.cand[nxt], w.ctr + kCtrCand + nxt, w.cnt_r[nxt], w.nc_cap, lane);
  }
}

template <typename T>
__device__ __noinline__ void verify_pass(const ScreenArgs<T>& a, const T* __restrict__ W,
                            const T* __restrict__ V, int nxt, double lamd, double (&v)[kParts],
                            int lane, int gwarp, int gwarps) {
  const int p = a.p, ld = a.ld;
  const ScreenWork<T>& w = a.w;
  const int nb = (p + kTile - 1) / kTile;
  const float lamf = (float)lamd;
  const T lam = (T)lamd;
  const int units = nb * nb * 4;
  // |a|, |b| < lambda / 2 (slightly less, covering the rounding of a + b)
  // decides the common case without floating-point work: |a + b| <= lambda,
  // so no failure, no candidate and a zero KKT term
  const unsigned small = mag_hi_below((T)(0.5 * lamd * (1.0 - 1e-6)));
  // the next sweep's screen keeps a margin below lambda (see kScreenMargin)
  const T lam_s = (T)(lamd * (1.0 - kScreenMargin));
  const unsigned small_s = mag_hi_below((T)(0.5 * lamd * (1.0 - kScreenMargin) * (1.0 - 1e-6)));
  for (int u = gwarp; u < units; u += gwarps) {
    const int tau = u >> 2, r0 = (u & 3) * 8;
    const int ta = tau / nb, tb = tau % nb;
    if (ta > tb) continue;
    const int j = tb * kTile + lane;
    const int i0 = ta * kTile + r0;
    if (i0 >= p) continue;
    const bool jv = j < p;
    T w1[8], v1[8], wt[8], vt[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      const bool ok = jv && i < p && i < j;
      w1[r] = ok ? __ldcg(W + (size_t)i * ld + j) : (T)0;
      v1[r] = ok ? __ldcg(V + (size_t)i * ld + j) : nan_t((T)0);
    }
    if (jv && i0 < j) {
      load8(W + (size_t)j * ld + i0, wt);
      load8(V + (size_t)j * ld + i0, vt);
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) wt[r] = vt[r] = (T)0;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      const bool pair = jv && i < p && i < j && !isnan(v1[r]);
      const bool vsmall = mag_hi(v1[r]) <= small && mag_hi(vt[r]) <= small;
      const bool wsmall = mag_hi(w1[r]) <= small_s && mag_hi(wt[r]) <= small_s;
      bool bad = false, next = false;
      if (pair && !vsmall) {
        const T x = ((T)0 - v1[r]) - vt[r];
        bad = fabs(x) - lam > (T)0;
      }
      push_list(bad, i, j, w.fail, w.ctr + kCtrFail, w.fail_cap, lane);
      if (pair && !wsmall) {
        const T x0 = ((T)0 - w1[r]) - wt[r];
        next = fabs(x0) - lam_s > (T)0;
      }
      push_cand(next, i, j, w.cand[nxt], w.ctr + kCtrCand + nxt, w.cnt_r[nxt], w.nc_cap, lane);
      if (pair && !wsmall) {
        // residual exactly 0 when |G| is below lambda by more than FP32
        // rounding; otherwise evaluated in FP64
        const float w1f = (float)w1[r], w2f = (float)wt[r];
        if (!(fabsf(w1f + w2f) <= lamf - 1e-5f * (1.0f + fabsf(w1f) + fabsf(w2f)))) {
          const double g = (double)w1[r] + (double)wt[r];
          v[kPartKkt] = fmax(v[kPartKkt], fmax(fabs(g) - lamd, 0.0));
          if (!isfinite(g)) v[kPartBad] += 1.0;
        }
      }
    }
  }
}

}  // namespace

template <typename T, bool MIXED>
__global__ void __launch_bounds__(kScreenThreads, 1) k_screened(const ScreenArgs<T> a) {
  using VT = Vec<T>;
  using VV = typename VT::V;
  constexpr int VN = VT::N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
  const int gwarp = blockIdx.x * nwarps + wid, gwarps = gridDim.x * nwarps;
  // per-candidate loops take threads (warps) in this order: consecutive
  // candidates land on different CTAs, so a few thousand candidates spread
  // their scattered loads over every SM's load pipeline
  const int sid = threadIdx.x * (int)gridDim.x + (int)blockIdx.x;
  const int swarp = wid * (int)gridDim.x + (int)blockIdx.x;
  const int p = a.p, P = a.P, ld = a.ld;
  const ScreenWork<T>& w = a.w;
  const WaitCtl& wc = a.wait;
  // the lambda being swept (the path's current one)
  int pk = a.path_n > 0 ? a.path_start : 0;
  double lamd = a.path_n > 0 ? a.path_lambda[pk] : a.lambda;
  T lam = (T)lamd;
  T lam_s = (T)(lamd * (1.0 - kScreenMargin));
  int tt = 0;  // sweeps of the whole launch (history rows)

  __shared__ double red[kScreenThreads / 32][kParts];
  __shared__ int s_tmp[32];
  __shared__ double s_res[kRes];
  __shared__ int s_stop;
  __shared__ unsigned long long s_dmax;  // the CTA's largest rowacc + D_i of the sweep (bits)
  __shared__ unsigned long long s_qmax;  // the same over the rows that stay quiet (bits)
  __shared__ int s_fill;                 // the CTA's largest pending fill the sweep would need
  __shared__ int s_fast;
  __shared__ double s_dsweep;
  __shared__ int s_nloud;
  extern __shared__ __align__(128) unsigned char dyn[];

  // the data checks of the kernels before this launch were not read by the
  // host yet: when one failed, end at once (every CTA reads the same word)
  if (a.input_flag != nullptr && ld_relaxed_s32(a.input_flag) != 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int k = 0; k < kRes; ++k) a.result[k] = 0.0;
      a.result[kResStatus] = 2.0;
      a.result[kResList] = -1.0;
    }
    return;
  }
  unsigned gen = 0;
  int where = 0;
  T* Wa = a.W;
  T* Wn = a.Wb;
  int cur = 0;
  int t = 0, first_delta = 0, since_best = 0;
  double best_kkt = 1e300;
  int status = -1;  // set when the launch ends early (overflow: kStatusDense)
  const bool kkt0 = a.kkt_only || a.n_sweeps <= 0;  // objective / KKT only
  int redo_total = 0;
  bool need_scan = true;  // row offsets of the current list still to be computed
  // lazy verification (see kLazySlack): bound accumulated on the pairs outside
  // the current list since it was screened, and whether the list's build is
  // kept from the previous sweep
  double acc = 0.0;
  bool reuse = false;
  // per-row form of the bound (w.rowacc): valid once every pair was screened
  // by this launch; force_full: a partial sweep could not keep all of its
  // new candidates, so the next sweep verifies everything
  bool rows_valid = a.start_list < 0 || kkt0;
  bool force_full = false;
  int n_lazy = 0, n_partial = 0;
  // deferred row updates: some stored rows of Wa lag behind their pending
  // entries (after a deferring sweep, until a flush)
  bool have_pend = false;

  // ---------------- screen the starting point (and its KKT for kkt_only);
  //                  the host zeroed the counters and row counts.  Or take
  //                  the list the previous launch left for its next sweep
  //                  (a superset screen of the same lambda: the verification
  //                  keeps the iterates exact whatever the list)
  if (a.start_list >= 0 && !kkt0) {
    cur = a.start_list;
    need_scan = a.start_scan != 0;  // else its row offsets and term count are in place
    acc = INFINITY;     // screened by another launch: the first sweep verifies
  } else {
    double v[kParts];
#pragma unroll
    for (int k = 0; k < kParts; ++k) v[k] = 0.0;
    screen_pass<T, MIXED>(a, Wa, cur, kkt0, lamd, v, lane, gwarp, gwarps);
    for (int i = gtid; i < p; i += gthreads) w.rowacc[i] = 0.0;
    if (kkt0) reduce_parts(v, a.partials, red);
    grid_barrier(a.barrier, gen, wc, ++where);
  }

  for (;;) {
    const bool do_sweep = !kkt0 && t < a.n_sweeps;
    double v[kParts];
#pragma unroll
    for (int k = 0; k < kParts; ++k) v[k] = 0.0;
    bool fast = false;       // this sweep skipped the verification (lazy)
    int mode = kModeFull;    // and (kModeDefer) its row pass
    int n_cur = 0;           // candidates of the sweep's list
    if (do_sweep) {
      int redo = 0;
      for (;;) {  // until the verification passes
        if (threadIdx.x == 0) {
          s_dmax = 0ull;
          s_qmax = 0ull;
          s_fill = 0;
        }
        const int N = ldi(w.ctr + kCtrCand + cur);
        n_cur = N;
        if (N > w.nc_cap || ld_relaxed_s32(wc.abort) != 0) {
          status = kStatusDense;
          break;
        }
        const int2* cand = w.cand[cur];
        // ---- build: row buckets of the current list (counted at the push),
        //      each row's candidates in colour-step order, and per candidate
        //      its record and correction terms (kept from the previous sweep
        //      when it reused its list: only the records are refreshed)
        if (!reuse) {
        if (need_scan) {  // else the previous sweep's reduce phase scanned the counts
          if (blockIdx.x == 0) {
            cta_scan([&](int k) { return ldi(w.cnt_r[cur] + k); }, p, w.off_r, w.cur_r, s_tmp,
                     w.ctr + kCtrTermsPred);
          }
          grid_barrier(a.barrier, gen, wc, ++where);
        }
        need_scan = true;
        if (ldi(w.ctr + kCtrTermsPred) > w.term_cap) {  // the terms cannot fit
          status = kStatusDense;
          break;
        }
        if (gtid == 0) w.ctr[kCtrTerms] = 0;  // allocated from two phases later
        for (int k = gtid; k < N; k += gthreads) {
          const int2 pr = __ldcg(cand + k);
          w.row_ent[atomicAdd(w.cur_r + pr.x, 1)] = k;
          w.row_ent[atomicAdd(w.cur_r + pr.y, 1)] = k;
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        // each row's candidates in colour-step order, one warp per row: the
        // steps of a row are distinct (a colour step pairs the row with one
        // partner), so a candidate's position is the number of smaller steps;
        // rows longer than the warp's buffer fall back to an insertion sort
        {
          int* sk = reinterpret_cast<int*>(dyn) + wid * 2 * kSortCap;
          int* ss = sk + kSortCap;
          for (int r = gwarp; r < p; r += gwarps) {
            const int b = ldi(w.off_r + r), e = ldi(w.off_r + r + 1), len = e - b;
            if (len <= kSortCap) {
              for (int x = lane; x < len; x += 32) {
                const int key = ldi(w.row_ent + b + x);
                const int2 kp = __ldcg(cand + key);
                sk[x] = key;
                ss[x] = pair_step(kp.x, kp.y, P);
              }
              __syncwarp();
              for (int x = lane; x < len; x += 32) {
                const int sx = ss[x];
                int rank = 0;
                for (int y = 0; y < len; ++y) rank += ss[y] < sx ? 1 : 0;
                const int key = sk[x];
                w.row_ent[b + rank] = key;
                if (__ldcg(cand + key).x == r)
                  w.nd_pi[key] = rank;
                else
                  w.nd_pj[key] = rank;
              }
              __syncwarp();
            } else if (lane == 0) {
              for (int x = b + 1; x < e; ++x) {
                const int key = ldi(w.row_ent + x);
                const int2 kp = __ldcg(cand + key);
                const int kc = pair_step(kp.x, kp.y, P);
                int y = x - 1;
                while (y >= b) {
                  const int2 yp = __ldcg(cand + ldi(w.row_ent + y));
                  if (pair_step(yp.x, yp.y, P) <= kc) break;
                  w.row_ent[y + 1] = ldi(w.row_ent + y);
                  --y;
                }
                w.row_ent[y + 1] = key;
              }
              for (int x = b; x < e; ++x) {
                const int k = ldi(w.row_ent + x);
                if (__ldcg(cand + k).x == r)
                  w.nd_pi[k] = x - b;
                else
                  w.nd_pj[k] = x - b;
              }
            }
          }
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        } else {
          need_scan = true;
        }
        // operands; each candidate's terms (row i's earlier candidates, then
        // row j's) get a contiguous range from a shared counter -- where the
        // range lies does not affect any value
        // (warp-uniform trips: a warp takes 32 consecutive candidates and
        // allocates their term ranges with one atomic)
        for (int k0 = swarp * 32; k0 < N; k0 += gwarps * 32) {
          const int k = k0 + lane;
          const bool valid = k < N;
          int i = 0, j = 0;
          if (valid) {
            const int2 pr = __ldcg(cand + k);
            i = pr.x;
            j = pr.y;
            T* rec = w.nd_rec + 4 * (size_t)k;
            T w1 = __ldcg(Wa + (size_t)i * ld + j), w2 = __ldcg(Wa + (size_t)j * ld + i);
            if (have_pend) {  // the rows' deferred updates, in order
              w1 = pend_fold(a, i, ldi(w.pend_n + i), j, w1);
              w2 = pend_fold(a, j, ldi(w.pend_n + j), i, w2);
            }
            rec[0] = w1;
            rec[1] = w2;
            rec[2] = __ldcg(a.Om + (size_t)i * ld + j);
            w.nd_delta[k] = (T)0;  // the fixed-point iteration starts from no change
            if (!reuse) rec[3] = a.sdiag[i] + a.sdiag[j];
          }
          if (reuse) continue;  // terms and s_ii + s_jj as the previous sweep built them
          const int bi = valid ? ldi(w.off_r + i) : 0, pi = valid ? ldi(w.nd_pi + k) : 0;
          const int bj = valid ? ldi(w.off_r + j) : 0, pj = valid ? ldi(w.nd_pj + k) : 0;
          const int cnt = pi + pj;
          int incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
          }
          int base = 0;
          if (lane == 31 && incl > 0) base = atomicAdd(w.ctr + kCtrTerms, incl);
          base = __shfl_sync(FULL, base, 31);
          int tp = base + incl - cnt;
          if (!valid) continue;
          w.term_ptr[k] = tp;
          if (tp + cnt > w.term_cap) continue;  // overflow: the sweep goes dense
          for (int m = 0; m < pi; ++m, ++tp) {
            const int q = ldi(w.row_ent + bi + m);
            const int2 qp = __ldcg(cand + q);
            const int u = qp.x == i ? qp.y : qp.x;
            w.term_pred[tp] = q;
            w.term_s[tp] = __ldg(a.S + (size_t)u * ld + j);
          }
          for (int m = 0; m < pj; ++m, ++tp) {
            const int q = ldi(w.row_ent + bj + m);
            const int2 qp = __ldcg(cand + q);
            const int u = qp.x == j ? qp.y : qp.x;
            w.term_pred[tp] = q;
            w.term_s[tp] = __ldg(a.S + (size_t)u * ld + i);
          }
        }
        if (gtid < kJacMax) w.jac[gtid] = 0;
        if (gtid == 0) w.ctr[kCtrLoud] = 0;
        if (gtid == 0) {
          w.ctr[kCtrJacDone] = 0;
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        if (ldi(w.ctr + kCtrTerms) > w.term_cap) {
          status = kStatusDense;
          break;
        }
        // ---- chain, in parallel: the changes d solve d_k = F_k(d of the
        //      earlier candidates sharing row i or j), a system over a DAG in
        //      colour-step order whose unique solution is the sequential
        //      walk's.  Iterating d <- F(d) from d = 0 over all candidates at
        //      once reaches it exactly: once an iteration leaves every d
        //      unchanged (bit for bit) the iterate satisfies the system.  Each
        //      link scales a perturbation by |s_uj| / (s_ii + s_jj), so the
        //      iteration settles after a few dozen rounds instead of one
        //      round per link.  Thread gtid owns candidate gtid (operands in
        //      registers); further candidates (N > threads) reload theirs.
        // only the CTAs that own candidates iterate (barrier among them);
        // the others wait at the phase's closing grid barrier.  Only the
        // first kJacThreads threads of a CTA own candidates (enough for one
        // candidate per thread over all SMs, at least two warps), so that
        // the rounds' scattered loads (and in FP64 the division of Eq. 3,
        // FP64 throughput per SM being small on this part) spread over the
        // SMs
        const int kJacThreads =
            min(kScreenThreads, max(64, ((N + (int)gridDim.x - 1) / (int)gridDim.x + 31) / 32 * 32));
        const int jac_ctas = min((int)gridDim.x, (N + kJacThreads - 1) / kJacThreads);
        const int jac_span = jac_ctas * kJacThreads;  // candidates owned one per thread
        if ((int)blockIdx.x < jac_ctas) {
          const int k0 = (int)threadIdx.x < kJacThreads ? (int)blockIdx.x * kJacThreads + (int)threadIdx.x
                                                      : N;
          const bool own = k0 < N;
          T w1 = (T)0, w2 = (T)0, om = (T)0, ss = (T)1;
          int t0 = 0, ts = 0, nt = 0;
          int tpr[4] = {0, 0, 0, 0};
          T tsv[4] = {(T)0, (T)0, (T)0, (T)0};
          if (own) {
            const T* rec = w.nd_rec + 4 * (size_t)k0;
            w1 = __ldcg(rec);
            w2 = __ldcg(rec + 1);
            om = __ldcg(rec + 2);
            ss = __ldcg(rec + 3);
            t0 = ldi(w.term_ptr + k0);
            const int pi = ldi(w.nd_pi + k0);
            ts = t0 + pi;
            nt = pi + ldi(w.nd_pj + k0);
#pragma unroll
            for (int x = 0; x < 4; ++x)
              if (x < nt) {
                tpr[x] = ldi(w.term_pred + t0 + x);
                tsv[x] = __ldcg(w.term_s + t0 + x);
              }
          }
          T dmine = (T)0;
          const T* dcur = w.nd_delta;
          T* dnext = w.nd_d2;
          for (int r = 0; r < kJacMax; ++r) {
            bool changed = false;
            if (own) {
              T vij = w1, vji = w2;
#pragma unroll
              for (int x = 0; x < 4; ++x)
                if (x < nt) {
                  const T d = __ldcg(dcur + tpr[x]);
                  if (d != (T)0) {
                    if (t0 + x < ts)
                      vij = fma_t(d, tsv[x], vij);
                    else
                      vji = fma_t(d, tsv[x], vji);
                  }
                }
              for (int x = 4; x < nt; ++x) {
                const T d = __ldcg(dcur + ldi(w.term_pred + t0 + x));
                if (d != (T)0) {
                  if (t0 + x < ts)
                    vij = fma_t(d, __ldcg(w.term_s + t0 + x), vij);
                  else
                    vji = fma_t(d, __ldcg(w.term_s + t0 + x), vji);
                }
              }
              const T xv = (ss * om - vij) - vji;
              const T sx = soft(xv, lam);
              T nw = (T)0;
              if (sx != (T)0) nw = sx / ss;
              const T delta = nw - om;
              changed = !same_bits(delta, dmine);
              dmine = delta;
              dnext[k0] = delta;
              w.nd_new[k0] = nw;
            }
            for (int k = k0 + jac_span; k < N; k += jac_span) {
              const T* rec = w.nd_rec + 4 * (size_t)k;
              const int u0 = ldi(w.term_ptr + k), us = u0 + ldi(w.nd_pi + k),
                        u1 = us + ldi(w.nd_pj + k);
              T vij = __ldcg(rec), vji = __ldcg(rec + 1);
              const T omk = __ldcg(rec + 2), ssk = __ldcg(rec + 3);
              for (int x = u0; x < u1; ++x) {
                const T d = __ldcg(dcur + ldi(w.term_pred + x));
                if (d != (T)0) {
                  if (x < us)
                    vij = fma_t(d, __ldcg(w.term_s + x), vij);
                  else
                    vji = fma_t(d, __ldcg(w.term_s + x), vji);
                }
              }
              const T xv = (ssk * omk - vij) - vji;
              const T sx = soft(xv, lam);
              T nw = (T)0;
              if (sx != (T)0) nw = sx / ssk;
              const T delta = nw - omk;
              changed |= !same_bits(delta, __ldcg(dcur + k));
              dnext[k] = delta;
              w.nd_new[k] = nw;
            }
            const bool moved = round_barrier_any(w.jac + r, (unsigned)jac_ctas, changed, wc,
                                                 ++where, (int)blockIdx.x);
            const T* tmp = dcur;
            dcur = dnext;
            dnext = const_cast<T*>(tmp);
            if (!moved) {
              // the solution sits in dcur; keep it in nd_delta
              if (dcur != w.nd_delta)
                for (int k = gtid; k < N; k += jac_ctas * (int)blockDim.x)
                  w.nd_delta[k] = __ldcg(dcur + k);
              if (gtid == 0) w.ctr[kCtrJacDone] = 1;
              break;
            }
          }
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        if (ldi(w.ctr + kCtrJacDone) == 0) {
          // not settled: nothing changed yet, the dense kernel takes the sweep
          status = kStatusDense;
          break;
        }
        // ---- reset the next list's counters
        if (gtid == 0) {
          w.ctr[kCtrCand + (1 - cur)] = 0;
          w.ctr[kCtrFail] = 0;
        }
        for (int k = gtid; k <= p; k += gthreads) w.cnt_r[1 - cur][k] = 0;
        // ---- diagonal (Eq. 2), one warp per row: W_ii after the row's
        //      pending updates and this sweep's changes (the dense kernel's FMA
        //      chain), the root in FP64, the diagonal's objective / KKT terms,
        //      the row's lazy-verification bound D_i, and tentatively the row's
        //      new pending entries (its changes in step order, then the
        //      diagonal change)
        // (one thread per row, rows spread over the CTAs: the row's loads are
        // a few dependent levels, so all rows proceed at once; the FMAs run
        // in the same order as the dense kernel's)
        for (int i = threadIdx.x * (int)gridDim.x + (int)blockIdx.x; i < p; i += gthreads) {
          const int b = ldi(w.off_r + i), ne = ldi(w.off_r + i + 1) - b;
          const int np = have_pend ? ldi(w.pend_n + i) : 0;
          int* pu = w.pend_u + (size_t)i * kPendRow;
          T* pdv = w.pend_d + (size_t)i * kPendRow;
          T wii = pend_fold(a, i, np, i, __ldcg(Wa + (size_t)i * ld + i));
          double dsum = 0.0;  // sum of |d| m_u over the row's changes
          int nchg = 0;
          for (int m0 = 0; m0 < ne; m0 += 8) {
            int qv[8];
            T dv[8], sv[8];
            int uv[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) qv[r] = m0 + r < ne ? ldi(w.row_ent + b + m0 + r) : -1;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              dv[r] = (T)0;
              uv[r] = 0;
              if (qv[r] >= 0) {
                const int2 qp = __ldcg(w.cand[cur] + qv[r]);
                uv[r] = qp.x == i ? qp.y : qp.x;
                dv[r] = __ldcg(w.nd_delta + qv[r]);
              }
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
              sv[r] = dv[r] != (T)0 ? __ldg(a.S + (size_t)uv[r] * ld + i) : (T)0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              if (dv[r] == (T)0) continue;
              dsum += fabs((double)dv[r]) * (double)__ldg(a.mrow + uv[r]);
              const int slot = np + nchg;
              if (slot < kPendRow) {
                pu[slot] = uv[r];
                pdv[slot] = dv[r];
              }
              ++nchg;
              wii = fma_t(dv[r], sv[r], wii);
            }
          }
          {
            const double sii = a.sdiag64[i];
            const T o_old = __ldcg(a.Om + (size_t)i * ld + i);
            const double oii = MIXED ? __ldcg(a.omdiag64 + i) : (double)o_old;
            const double ci = (double)wii - oii * sii;
            const double nw = (-ci + sqrt(ci * ci + 4.0 * sii)) / (2.0 * sii);
            w.diag_old[i] = o_old;
            if (MIXED) w.omdiag_old[i] = oii;
            w.diag_new[i] = nw;
            const T dd = (T)(nw - oii);
            w.diag_dd[i] = dd;
            const double dd64 = fabs(nw - oii);
            v[kPartDelta] = fmax(v[kPartDelta], dd64);
            // objective / KKT terms of the diagonal after the sweep
            const T wend = dd != (T)0 ? fma_t(dd, __ldg(a.S + (size_t)i * ld + i), wii) : wii;
            const double wd = (double)wend;
            const double od = MIXED ? nw : (double)(T)nw;
            if (od > 0.0 && isfinite(wd) && isfinite(od)) {
              v[kPartKkt] = fmax(v[kPartKkt], fabs(wd - 1.0 / od));
              v[kPartQuad] += od * wd;
              v[kPartLog] += log(od);
            } else {
              v[kPartBad] += 1.0;
            }
            const double di = dsum + dd64 * (double)__ldg(a.mrow + i);
            // the row's bound since its pairs were screened, and whether it
            // leaves half the margin (its pairs then need a verification)
            const double ai = rows_valid ? __ldcg(w.rowacc + i) + di : INFINITY;
            const bool is_loud = !(ai <= 0.5 * (kScreenMargin - kLazySlack) * lamd);
            w.rowa_new[i] = ai;
            w.loudf[i] = is_loud ? 1 : 0;
            if (is_loud) {
              const int slot = atomicAdd(w.ctr + kCtrLoud, 1);
              if (slot < kLoudMax) w.loud[slot] = i;
            } else {
              atomicMax(&s_qmax, (unsigned long long)__double_as_longlong(ai));
            }
            if (rows_valid) atomicMax(&s_dmax, (unsigned long long)__double_as_longlong(ai));
            int need = np + nchg;
            if (dd != (T)0) {
              if (need < kPendRow) {
                pu[need] = i;
                pdv[need] = dd;
              }
              ++need;
            }
            w.pend_new[i] = need;
            atomicMax(&s_fill, need);
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          w.dpart[blockIdx.x] = __longlong_as_double((long long)s_dmax);
          w.apart[blockIdx.x] = __longlong_as_double((long long)s_qmax);
          w.dfill[blockIdx.x] = s_fill;
        }
        // ---- commit the candidates' new values (both triangles)
        for (int k = sid; k < N; k += gthreads) {
          const T d = __ldcg(w.nd_delta + k);
          if (d != (T)0) {
            const int2 pr = __ldcg(cand + k);
            const T nw = __ldcg(w.nd_new + k);
            a.Om[(size_t)pr.x * ld + pr.y] = nw;
            a.Om[(size_t)pr.y * ld + pr.x] = nw;
            v[kPartDelta] = fmax(v[kPartDelta], (double)fabs(d));
            v[kPartActive] += 2.0;  // counted per owner, as the dense pass does
          }
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        // ---- lazy verification: every CTA forms the same decision.  A pair
        //      outside the list has moved by at most rowacc_i + rowacc_j (+
        //      this sweep's D_i + D_j) since it was screened.  LAZY (every
        //      row within half the margin): row pass without V, no
        //      verification, the list stays.  DEFER (the same, and every
        //      row's pending entries fit): no row pass either; the rows'
        //      changes and diagonal changes stay pending on the stored W.
        //      PARTIAL (a few rows beyond half the margin, the entries fit):
        //      as DEFER, and the pairs of those rows are verified and
        //      screened (partial_verify).  FULL: row pass with V,
        //      verification, fresh screen
        if (threadIdx.x == 0) {
          double dm = 0.0, qm = 0.0;
          int fm = 0;
          for (int c = 0; c < (int)gridDim.x; ++c) {
            dm = fmax(dm, __ldcg(w.dpart + c));
            qm = fmax(qm, __ldcg(w.apart + c));
            fm = max(fm, ldi(w.dfill + c));
          }
          const int nl = ldi(w.ctr + kCtrLoud);
          const bool may = a.lazy_verify && rows_valid && !force_full;
          const bool all_quiet = may && nl == 0;
          const bool partial = may && nl > 0 && nl <= kLoudMax && fm <= kPendRow;
          s_fast = all_quiet ? (fm <= kPendRow ? kModeDefer : kModeLazy)
                             : (partial ? kModePartial : kModeFull);
          // largest rowacc after the sweep (verified rows restart from 0)
          s_dsweep = partial ? qm : dm;
          s_nloud = nl;
        }
        __syncthreads();
        mode = s_fast;
        fast = mode != kModeFull;
        const bool full = mode == kModeFull;
        const bool deferred = mode == kModeDefer || mode == kModePartial;
        if (mode == kModeDefer) {
          for (int i = gtid; i < p; i += gthreads) w.pend_n[i] = ldi(w.pend_new + i);
        } else if (mode == kModePartial) {
          // pend_n still counts the old entries: the verification reads the
          // rows at the visit; the counts advance once the sweep stands
        } else {
          if (have_pend) {  // the stored rows catch up before the row pass reads them
            flush_pending(a, Wa, lane, gwarp, gwarps);
            grid_barrier(a.barrier, gen, wc, ++where);
            for (int i = gtid; i < p; i += gthreads) w.pend_n[i] = 0;
            have_pend = false;
          }
          // ---- rows: W after the colour steps, W += dw S_i, V (FULL)
          {
            int* l_u = reinterpret_cast<int*>(dyn) + wid * kRowList * 2;
            int* l_c = l_u + kRowList;
            T* l_d = reinterpret_cast<T*>(reinterpret_cast<int*>(dyn) + nwarps * kRowList * 2) +
                     wid * kRowList;
            // two work items per row, one per half of its columns (vectors
            // [0, nv/2) and [nv/2, nv)), so rows spread evenly over the warps
            const int nv = ld / VN;
            for (int item = gwarp; item < 2 * p; item += gwarps) {
              const int i = item >> 1, half = item & 1;
              const int qbeg = half ? nv / 2 : 0, qend = half ? nv : nv / 2;
              const int cbeg = qbeg * VN, cend = qend * VN;  // the half's columns
              const int b = ldi(w.off_r + i), ne = ldi(w.off_r + i + 1) - b;
              // the row's first candidate partners (lane m < 32, for the V marks
              // below) and the diagonal change the diagonal pass formed
              int my_u = -1;
              if (lane < ne) {
                const int2 qp = __ldcg(w.cand[cur] + ldi(w.row_ent + b + lane));
                my_u = qp.x == i ? qp.y : qp.x;
              }
              const T dd = __ldcg(w.diag_dd + i);
              // the row's changes in step order, in chunks of kRowList
              const T* Srow = a.S + (size_t)i * ld;
              int c_last = -1;  // step of the last change of the previous chunks
              int done = 0;
              bool first = true;
              do {
                int cnt = 0;
                int m0 = done;
                // compact the next changes (d != 0) into the warp's list
                while (m0 < ne && cnt < kRowList) {
                  const int m = m0 + lane;
                  int q = -1;
                  T d = (T)0;
                  if (m < ne) {
                    q = ldi(w.row_ent + b + m);
                    d = __ldcg(w.nd_delta + q);
                  }
                  const bool nz = m < ne && d != (T)0;
                  const unsigned bal = __ballot_sync(FULL, nz);
                  const int room = kRowList - cnt;
                  // take whole 32-entry groups only when they fit
                  if (__popc(bal) > room) break;
                  if (nz) {
                    const int slot = cnt + __popc(bal & ((1u << lane) - 1u));
                    const int2 qp = __ldcg(w.cand[cur] + q);
                    const int u = qp.x == i ? qp.y : qp.x;
                    l_u[slot] = u;
                    l_c[slot] = pair_step(min(i, u), max(i, u), P);
                    l_d[slot] = d;
                  }
                  cnt += __popc(bal);
                  m0 = min(ne, m0 + 32);
                }
                __syncwarp();
                const bool last = m0 >= ne;
                const T* src = (first ? Wa : Wn) + (size_t)i * ld;
                // U 16-byte vectors per lane per iteration; lane l takes vectors
                // q0 + 32 u, u < U (two, so that the paired S-row loads below fit
                // in registers)
                constexpr int U = 2;
                for (int q0 = qbeg + lane; q0 < qend; q0 += 32 * U) {
                  T acc[U][VN], vv[U][VN];
                  int cx[U][VN];
                  bool cap[U][VN];  // V captured (in this chunk or an earlier one)
  #pragma unroll
                  for (int uu = 0; uu < U; ++uu) {
                    const int q = q0 + 32 * uu;
                    if (q < qend)
                      VT::split(__ldcg(reinterpret_cast<const VV*>(src) + q), acc[uu]);
                    else
  #pragma unroll
                      for (int e = 0; e < VN; ++e) acc[uu][e] = (T)0;
  #pragma unroll
                    for (int e = 0; e < VN; ++e) {
                      const int x = q * VN + e;
                      cx[uu][e] = (x < p && x != i) ? pair_step(min(i, x), max(i, x), P) : 0x7fffffff;
                      cap[uu][e] = c_last >= cx[uu][e];
                      vv[uu][e] = (T)0;
                    }
                  }
                  // the diagonal's S row (last chunk) and the changes' S rows two
                  // at a time are requested before their values are used, so
                  // each lane keeps several independent loads in flight
                  T si[U][VN];
                  if (last && dd != (T)0) {
  #pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                      const int q = q0 + 32 * uu;
                      if (q < qend) VT::split(__ldg(reinterpret_cast<const VV*>(Srow) + q), si[uu]);
                    }
                  }
                  auto load_row = [&](int u, T (&sv)[U][VN]) {
                    const VV* su = reinterpret_cast<const VV*>(a.S + (size_t)u * ld);
  #pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                      const int q = q0 + 32 * uu;
                      if (q < qend) VT::split(__ldg(su + q), sv[uu]);
                      else
  #pragma unroll
                        for (int e = 0; e < VN; ++e) sv[uu][e] = (T)0;
                    }
                  };
                  auto apply = [&](int cm, T d, const T (&sv)[U][VN]) {
  #pragma unroll
                    for (int uu = 0; uu < U; ++uu)
  #pragma unroll
                      for (int e = 0; e < VN; ++e) {
                        // V: W before the first change at or after the pair's step
                        if (!cap[uu][e] && cm >= cx[uu][e]) {
                          vv[uu][e] = acc[uu][e];
                          cap[uu][e] = true;
                        }
                        acc[uu][e] = fma_t(d, sv[uu][e], acc[uu][e]);
                      }
                  };
                  int m = 0;
                  for (; m + 1 < cnt; m += 2) {
                    T sa[U][VN], sb[U][VN];
                    load_row(l_u[m], sa);
                    load_row(l_u[m + 1], sb);
                    apply(l_c[m], l_d[m], sa);
                    apply(l_c[m + 1], l_d[m + 1], sb);
                  }
                  if (m < cnt) {
                    T sa[U][VN];
                    load_row(l_u[m], sa);
                    apply(l_c[m], l_d[m], sa);
                  }
  #pragma unroll
                  for (int uu = 0; uu < U; ++uu) {
                    const int q = q0 + 32 * uu;
                    if (q >= qend) continue;
                    T out[VN];
                    T* vrow = a.V + (size_t)i * ld + q * VN;
  #pragma unroll
                    for (int e = 0; e < VN; ++e) {
                      // not captured: every change so far precedes the pair's step
                      if (!cap[uu][e]) vv[uu][e] = acc[uu][e];
                      out[e] = (last && dd != (T)0) ? fma_t(dd, si[uu][e], acc[uu][e]) : acc[uu][e];
                      if (full && c_last < cx[uu][e]) vrow[e] = vv[uu][e];
                    }
                    reinterpret_cast<VV*>(Wn + (size_t)i * ld)[q] = VT::join(out);
                  }
                }
                if (cnt > 0) c_last = l_c[cnt - 1];
                __syncwarp();
                first = false;
                done = m0;
                if (last) break;
              } while (true);
              // candidates of this row (changed or not) and the diagonal are not verified
              __syncwarp();
              if (!full) continue;
              if (ne <= 32) {
                if (my_u >= cbeg && my_u < cend) a.V[(size_t)i * ld + my_u] = nan_t((T)0);
              } else {
                for (int m = lane; m < ne; m += 32) {
                  const int2 qp = __ldcg(w.cand[cur] + ldi(w.row_ent + b + m));
                  const int u = qp.x == i ? qp.y : qp.x;
                  if (u >= cbeg && u < cend) a.V[(size_t)i * ld + u] = nan_t((T)0);
                }
              }
              if (lane == 0 && i >= cbeg && i < cend) a.V[(size_t)i * ld + i] = nan_t((T)0);
              __syncwarp();
            }
          }
          grid_barrier(a.barrier, gen, wc, ++where);
        }
        // ---- the new diagonal
        for (int k = gtid; k < p; k += gthreads) {
          const double nw = __ldcg(w.diag_new + k);
          a.Om[(size_t)k * ld + k] = (T)nw;
          if (MIXED) a.omdiag64[k] = nw;
        }
        // ---- verify the other pairs; objective / KKT; screen the next sweep
        //      (FULL only: otherwise none of them can have reached the
        //      threshold, their KKT terms are zero, and the list stays)
        if (full) verify_pass<T>(a, Wn, a.V, 1 - cur, lamd, v, lane, gwarp, gwarps);
        if (mode == kModePartial) partial_verify<T>(a, Wa, cur, s_nloud, lamd, v, lane, swarp, gwarps);
        // the candidates' own terms (and their screen: every nonzero stays a
        // candidate); warp-uniform trip count for the list pushes.  Their W
        // after the sweep: the row pass's rows, or (DEFER) the stored rows
        // with the pending entries
        for (int k0 = swarp * 32; k0 < N; k0 += gwarps * 32) {
          const int k = k0 + lane;
          bool next = false;
          int i = 0, j = 0;
          if (k < N) {
            const int2 pr = __ldcg(cand + k);
            i = pr.x;
            j = pr.y;
            const T d = __ldcg(w.nd_delta + k);
            const T omk = d != (T)0 ? __ldcg(w.nd_new + k) : __ldcg(w.nd_rec + 4 * (size_t)k + 2);
            T w1, w2;
            if (deferred) {
              w1 = pend_fold(a, i, ldi(w.pend_new + i), j, __ldcg(Wa + (size_t)i * ld + j));
              w2 = pend_fold(a, j, ldi(w.pend_new + j), i, __ldcg(Wa + (size_t)j * ld + i));
            } else {
              w1 = __ldcg(Wn + (size_t)i * ld + j);
              w2 = __ldcg(Wn + (size_t)j * ld + i);
            }
            const double om = (double)omk, g = (double)w1 + (double)w2;
            next = omk != (T)0 || (fabs(((T)0 - w1) - w2) - lam_s > (T)0);
            v[kPartKkt] = fmax(v[kPartKkt], kkt_offdiag(om, g, lamd));
            v[kPartQuad] += om * g;
            v[kPartPen] += fabs(om);
            if (!isfinite(g) || !isfinite(om)) v[kPartBad] += 1.0;
          }
          push_cand(next && !fast, i, j, w.cand[1 - cur], w.ctr + kCtrCand + 1 - cur,
                    w.cnt_r[1 - cur], w.nc_cap, lane);
        }
        grid_barrier(a.barrier, gen, wc, ++where);
        const int nf = ldi(w.ctr + kCtrFail);
        if (nf == 0) break;
        // ---- undo the sweep, add the failing pairs, redo
        for (int k = gtid; k < N; k += gthreads) {
          if (__ldcg(w.nd_delta + k) != (T)0) {
            const int2 pr = __ldcg(cand + k);
            const T om = __ldcg(w.nd_rec + 4 * (size_t)k + 2);
            a.Om[(size_t)pr.x * ld + pr.y] = om;
            a.Om[(size_t)pr.y * ld + pr.x] = om;
          }
        }
        for (int i = gtid; i < p; i += gthreads) {
          a.Om[(size_t)i * ld + i] = __ldcg(w.diag_old + i);
          if (MIXED) a.omdiag64[i] = __ldcg(w.omdiag_old + i);
        }
        const int add = min(min(nf, w.fail_cap), w.nc_cap - N);
        for (int f = gtid; f < add; f += gthreads) {
          const int2 pr = __ldcg(w.fail + f);
          w.cand[cur][N + f] = pr;
          atomicAdd(w.cnt_r[cur] + pr.x, 1);
          atomicAdd(w.cnt_r[cur] + pr.y, 1);
        }
        if (gtid == 0) {
          w.ctr[kCtrCand + cur] = N + add;
          w.ctr[kCtrFail] = 0;
        }
#pragma unroll
        for (int k = 0; k < kParts; ++k) v[k] = 0.0;
        ++redo_total;
        reuse = false;  // the list grew: build it again
        grid_barrier(a.barrier, gen, wc, ++where);
        if (add < min(nf, w.fail_cap) || ++redo > a.max_redo) {
          status = kStatusDense;
          break;
        }
      }
      if (status == kStatusDense) {
        // nothing of this sweep was kept; report the state as it stands
        break;
      }
      reduce_parts(v, a.partials, red);
      // the per-row bounds after the sweep: 0 after a full verification,
      // and for the rows a partial one verified; else grown by D_i
      for (int i = gtid; i < p; i += gthreads)
        w.rowacc[i] = (mode == kModeFull || (mode == kModePartial && ldi(w.loudf + i) != 0))
                          ? 0.0
                          : __ldcg(w.rowa_new + i);
      bool grew = false;
      if (mode == kModePartial) {
        // the sweep stands: its pending entries count, and the pairs it
        // screened join the kept list (a list that cannot take them all
        // makes the next sweep a full one)
        for (int i = gtid; i < p; i += gthreads) w.pend_n[i] = ldi(w.pend_new + i);
        const int pushed = ldi(w.ctr + kCtrCand + 1 - cur);
        const int add = min(min(pushed, w.nc_cap), w.nc_cap - n_cur);
        for (int f = gtid; f < add; f += gthreads) {
          const int2 pr = __ldcg(w.cand[1 - cur] + f);
          w.cand[cur][n_cur + f] = pr;
          atomicAdd(w.cnt_r[cur] + pr.x, 1);
          atomicAdd(w.cnt_r[cur] + pr.y, 1);
        }
        if (gtid == 0) w.ctr[kCtrCand + cur] = n_cur + add;
        grew = pushed > 0;
        force_full = add < pushed;
      } else {
        force_full = false;
      }
      if (mode == kModeFull) rows_valid = true;
      // row offsets of the next sweep's list (its pushes are complete); a
      // lazy sweep keeps its list, offsets and build
      if (blockIdx.x == 0 && !fast) {
        cta_scan([&](int k) { return ldi(w.cnt_r[1 - cur] + k); }, p, w.off_r, w.cur_r, s_tmp,
                 w.ctr + kCtrTermsPred);
      }
      if (blockIdx.x == 0 && fast)  // fresh cursors for a later build of the kept list
        for (int k = threadIdx.x; k <= p; k += blockDim.x) w.cur_r[k] = ldi(w.off_r + k);
      need_scan = grew;  // a grown list is counted again by the next build
      acc = fast ? 2.0 * s_dsweep : 0.0;
      reuse = fast && !grew;
      n_lazy += fast ? 1 : 0;
      n_partial += mode == kModePartial ? 1 : 0;
      if (mode == kModeDefer || mode == kModePartial) have_pend = true;
      grid_barrier(a.barrier, gen, wc, ++where);
    }

    // ---------------- every CTA reduces the partials identically (warp 0:
    //                  lanes stride over the CTAs, then a fixed shuffle tree)
    double kkt = 0.0, quad = 0.0, pen = 0.0, lg = 0.0, dl = 0.0, ac = 0.0, bad = 0.0;
    if (wid == 0) {
      for (int b = lane; b < (int)gridDim.x; b += 32) {
        const double* q = a.partials + (size_t)b * kParts;
        kkt = fmax(kkt, __ldcg(q + kPartKkt));
        quad += __ldcg(q + kPartQuad);
        pen += __ldcg(q + kPartPen);
        lg += __ldcg(q + kPartLog);
        dl = fmax(dl, __ldcg(q + kPartDelta));
        ac += __ldcg(q + kPartActive);
        bad += __ldcg(q + kPartBad);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        kkt = fmax(kkt, __shfl_xor_sync(FULL, kkt, o));
        dl = fmax(dl, __shfl_xor_sync(FULL, dl, o));
        quad += __shfl_xor_sync(FULL, quad, o);
        pen += __shfl_xor_sync(FULL, pen, o);
        lg += __shfl_xor_sync(FULL, lg, o);
        ac += __shfl_xor_sync(FULL, ac, o);
        bad += __shfl_xor_sync(FULL, bad, o);
      }
    }
    if (threadIdx.x == 0) {
      const double obj = -lg + 0.5 * quad + lamd * pen;
      const bool aborted = ld_relaxed_s32(wc.abort) != 0;
      const bool nonfinite = bad > 0.0 || !isfinite(obj) || !isfinite(kkt);
      const int sweeps_done = do_sweep ? t + 1 : t;
      if (do_sweep && first_delta == 0 && dl < a.delta_tol) first_delta = sweeps_done;
      const bool conv = (a.stop_rule == 1) ? (do_sweep && dl < a.tol) : (kkt <= a.tol);
      bool stalled = false;
      if (do_sweep) {
        if (kkt < 0.9 * best_kkt) {
          best_kkt = kkt;
          since_best = 0;
        } else if (++since_best >= 4 && a.stall_stop) {
          stalled = true;
        }
      }
      // the next sweep's candidates overflowed: hand over to the dense kernel
      const bool dense_next = !fast && ldi(w.ctr + kCtrCand + (1 - cur)) > w.nc_cap;
      s_res[kResSweeps] = sweeps_done;
      s_res[kResKkt] = kkt;
      s_res[kResObj] = obj;
      s_res[kResDelta] = dl;
      s_res[kResActive] = ac * 0.5;
      s_res[kResFirstDelta] = first_delta;
      s_res[kResRedo] = redo_total;
      s_res[kResPath] = pk;
      s_res[kResLazy] = n_lazy;
      s_res[kResAcc] = acc;  // the lazy bound accumulated on the next sweep's list
      s_res[kResPartial] = n_partial;
      s_res[kResList] = (do_sweep && !aborted && !nonfinite && !dense_next)
                            ? (double)(fast ? cur : 1 - cur)
                            : -1.0;
      s_res[kResStatus] = aborted      ? 3.0
                          : nonfinite  ? 2.0
                          : conv       ? 0.0
                          : stalled    ? 4.0
                          : (dense_next && sweeps_done < a.n_sweeps && !kkt0)
                              ? (double)kStatusDense
                              : 1.0;
      s_stop = (aborted || nonfinite || conv || stalled || kkt0 ||
                sweeps_done >= a.n_sweeps || dense_next)
                   ? 1
                   : 0;
      if (blockIdx.x == 0) {
        if (do_sweep && tt < a.hist_len) {
          double* h = a.hist + (size_t)tt * kHist;
          h[0] = dl;
          h[1] = kkt;
          h[2] = obj;
          h[3] = ac * 0.5;
        }
        if (s_stop) {
          for (int k = 0; k < kRes; ++k) a.result[k] = s_res[k];
          if (a.path_n > 0)
            for (int k = 0; k < kRes; ++k) a.path_res[(size_t)pk * kRes + k] = s_res[k];
        }
      }
    }
    __syncthreads();
    if (kkt0) break;
    // the accepted sweep's W becomes current (a deferring sweep left its
    // updates pending on the stored rows)
    if (mode != kModeDefer && mode != kModePartial) {
      T* tmp = Wa;
      Wa = Wn;
      Wn = tmp;
    }
    if (!fast) cur = 1 - cur;
    if (do_sweep) ++tt;
    if (s_stop) {
      // lambda path: on to the next lambda unless this one ended in an error
      // or needs the dense kernel
      const int code = (int)s_res[kResStatus];
      if (a.path_n == 0 || pk + 1 >= a.path_n || code == 2 || code == 3 || code == kStatusDense ||
          (code == 4 && a.path_break_stall))
        break;
      // this lambda's Omega (copy and / or support count), the next lambda's
      // screen from scratch
      if (a.path_om) {
        T* out = a.path_om + (size_t)pk * p * a.path_ldo;
        for (size_t e = gtid; e < (size_t)p * p; e += gthreads) {
          const int r = (int)(e / p), c = (int)(e % p);
          out[(size_t)r * a.path_ldo + c] = __ldcg(a.Om + (size_t)r * ld + c);
        }
      }
      if (a.path_cnt) {
        float* cnt = a.path_cnt + (size_t)pk * p * p;
        for (size_t e = gtid; e < (size_t)p * p; e += gthreads) {
          const int r = (int)(e / p), c = (int)(e % p);
          if (__ldcg(a.Om + (size_t)r * ld + c) != (T)0) atomicAdd(cnt + e, 1.0f);
        }
      }
      ++pk;
      lamd = a.path_lambda[pk];
      lam = (T)lamd;
      lam_s = (T)(lamd * (1.0 - kScreenMargin));
      t = 0;
      first_delta = 0;
      since_best = 0;
      best_kkt = 1e300;
      if (gtid == 0) w.ctr[kCtrCand + cur] = 0;
      for (int k = gtid; k <= p; k += gthreads) w.cnt_r[cur][k] = 0;
      if (have_pend) {  // the screen reads the true W
        flush_pending(a, Wa, lane, gwarp, gwarps);
        grid_barrier(a.barrier, gen, wc, ++where);
        for (int i = gtid; i < p; i += gthreads) w.pend_n[i] = 0;
        have_pend = false;
      }
      grid_barrier(a.barrier, gen, wc, ++where);
      {
        double vz[kParts];
#pragma unroll
        for (int k = 0; k < kParts; ++k) vz[k] = 0.0;
        screen_pass<T, MIXED>(a, Wa, cur, false, lamd, vz, lane, gwarp, gwarps);
      }
      for (int i = gtid; i < p; i += gthreads) w.rowacc[i] = 0.0;
      rows_valid = true;
      force_full = false;
      need_scan = true;
      acc = 0.0;  // a fresh screen of the current iterate
      reuse = false;
      grid_barrier(a.barrier, gen, wc, ++where);
      continue;
    }
    ++t;
  }
  // the last lambda's Omega (path)
  if (a.path_n > 0 && status != kStatusDense && (int)s_res[kResStatus] != 2 &&
      (int)s_res[kResStatus] != 3 && !((int)s_res[kResStatus] == 4 && a.path_break_stall)) {
    if (a.path_om) {
      T* out = a.path_om + (size_t)pk * p * a.path_ldo;
      for (size_t e = gtid; e < (size_t)p * p; e += gthreads) {
        const int r = (int)(e / p), c = (int)(e % p);
        out[(size_t)r * a.path_ldo + c] = __ldcg(a.Om + (size_t)r * ld + c);
      }
    }
    if (a.path_cnt) {
      float* cnt = a.path_cnt + (size_t)pk * p * p;
      for (size_t e = gtid; e < (size_t)p * p; e += gthreads) {
        const int r = (int)(e / p), c = (int)(e % p);
        if (__ldcg(a.Om + (size_t)r * ld + c) != (T)0) atomicAdd(cnt + e, 1.0f);
      }
    }
  }

  if (status == kStatusDense && blockIdx.x == 0 && threadIdx.x == 0) {
    // the sweep in progress was undone or never started: t sweeps are done
    // (for a path: of lambda pk, whose index the host reads from kResPath)
    a.result[kResPath] = pk;
    a.result[kResSweeps] = t;
    a.result[kResKkt] = t > 0 ? s_res[kResKkt] : 1e300;
    a.result[kResObj] = t > 0 ? s_res[kResObj] : 0.0;
    a.result[kResDelta] = t > 0 ? s_res[kResDelta] : 0.0;
    a.result[kResActive] = t > 0 ? s_res[kResActive] : 0.0;
    a.result[kResFirstDelta] = first_delta;
    a.result[kResRedo] = redo_total;
    a.result[kResList] = -1.0;
    a.result[kResStatus] = ld_relaxed_s32(wc.abort) != 0 ? 3.0 : (double)kStatusDense;
  }
  // deferred updates into the stored rows, unless the host rebuilds W itself
  // (a dense hand-over always needs them)
  if (have_pend && (a.keep_w || status == kStatusDense)) {
    flush_pending(a, Wa, lane, gwarp, gwarps);
    grid_barrier(a.barrier, gen, wc, ++where);
  }
  // leave W in the caller's buffer
  if (Wa != a.W) {
    const size_t n = (size_t)p * ld / VN;
    const VV* s = reinterpret_cast<const VV*>(Wa);
    VV* d = reinterpret_cast<VV*>(a.W);
    for (size_t k = gtid; k < n; k += gthreads) d[k] = __ldcg(s + k);
  }
}

size_t screened_dyn_smem(bool mixed) {
  // per warp: the row pass's staged changes (partner, step, delta), or (in
  // another phase) the row sort's keys and steps
  const size_t rows = (size_t)kRowList * (8 + (mixed ? 4 : 8));
  const size_t sort = (size_t)2 * kSortCap * sizeof(int);
  return (size_t)(kScreenThreads / 32) * (rows > sort ? rows : sort);
}

template <typename T, bool MIXED>
cudaError_t launch_screened_impl(const ScreenArgs<T>& a, int grid, cudaStream_t st) {
  const size_t dyn = screened_dyn_smem(MIXED);
  const void* fn = (const void*)k_screened<T, MIXED>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  note_launches(1);
  void* kargs[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kScreenThreads), kargs, dyn, st);
}

cudaError_t launch_screened(const ScreenArgs<double>& a, int grid, cudaStream_t st) {
  return launch_screened_impl<double, false>(a, grid, st);
}
cudaError_t launch_screened(const ScreenArgs<float>& a, int grid, cudaStream_t st) {
  return launch_screened_impl<float, true>(a, grid, st);
}

cudaError_t screened_occupancy(bool mixed, int* blocks_per_sm) {
  const size_t dyn = screened_dyn_smem(mixed);
  const void* fn = mixed ? (const void*)k_screened<float, true> : (const void*)k_screened<double, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  return mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_screened<float, true>,
                                                              kScreenThreads, dyn)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     blocks_per_sm, k_screened<double, false>, kScreenThreads, dyn);
}

}  // namespace concord
