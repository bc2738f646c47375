// Sparse FP64 polish of a mixed-precision solve (sm_103a).
//
// After the FP32 sweeps the iterate is close to the solution and every pair
// that can still change is in the FP32 phase's last candidate list (pairs
// with omega_ij != 0 or |G_ij| > 0.9 lambda when it was screened, G = W +
// W^T).  The lazy-verification argument of the screened kernel bounds how
// far G of a pair outside the list can move: by 2 max_i D_i per sweep, with
// D_i = sum of |d| m_u over the row's changes plus |dw| m_i (m_u =
// max_{x != u} |s_ux|).  Moving from the FP32 S to the FP64 S (the refined
// entries, and FP32 rounding) adds at most 2 max_i ||Omega_i||_1 max|dS|.
// While the sum stays within (kScreenMargin - kLazySlack) lambda, no pair
// outside the list reaches the threshold, so the FP64 sweeps change only the
// candidates, and the KKT terms of all other pairs are zero.  Then no sweep
// needs W as a whole: each W entry it reads is a sum over the nonzeros of a
// row of Omega,
//   W_ij = omega_ii s_ij + sum_{u in N(i)} omega_iu s_uj,
// so the polish runs on the candidates alone, without the O(p^2) rebuild of
// W in FP64 and without the p^2 row and verification passes.
//
// One sweep (Section 3.2, Algorithm 1; Eq. 3 and Eq. 2 written as the direct
// sums of their definitions over the nonzeros):
//   base     per candidate (i, j): a1 = sum_{u != j} omega_iu s_uj and
//            a2 = sum_{u != i} omega_ju s_ui from the values at the sweep's
//            start;
//   chain    the changes d solve d_k = F_k(d of the candidates of rows i and
//            j visited earlier), F_k = Eq. 3 with a1 += d_(i,u) s_uj over
//            the earlier (i, u) (and likewise a2).  Fixed-point rounds from
//            d = 0 until a round changes no d bit for bit: such an iterate
//            satisfies every equation, so it is the sequential solution;
//   diagonal Eq. 2 per row with the new off-diagonal values, the row bound
//            D_i, and the diagonal's objective / KKT terms;
//   decision the bound is kept per row (rowa_i: pair bound rowa_i + rowa_j,
//            from the FP32 phase's per-row bound plus the change of S).
//            Rows beyond half the margin have their pairs verified exactly
//            (their W entries are short sums too); too many such rows or a
//            pair that would leave zero: nothing is committed and the launch
//            returns kStatusNeedW (the host then rebuilds W and runs the
//            screened polish, which verifies everything);
//   terms    objective and KKT terms of the candidates after the sweep.
// Each candidate row's entries are kept in colour-step order; every sum runs
// in a fixed order, so the iterates do not depend on the launch layout.
#include "kernels.h"

namespace concord {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWarps = kPolishThreads / 32;
constexpr int kSortCap = 256;  // row entries whose steps a warp stages in shared memory
constexpr int kQ = 4;          // terms per side of a thread's first candidate kept in registers

__device__ __forceinline__ int other_end(int2 pr, int r) { return pr.x == r ? pr.y : pr.x; }

__device__ __forceinline__ void atomic_max_nonneg(int* slot, double v) {
  // nonnegative doubles order as their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double ld_nonneg(const int* slot) {
  return __longlong_as_double((long long)__ldcg(reinterpret_cast<const unsigned long long*>(slot)));
}

// Largest value over the CTA (every thread passes its own; thread 0 gets it).
__device__ __forceinline__ double block_max(double v, double* s_w) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kWarps; ++k) m = fmax(m, s_w[k]);
  return m;
}

// Exclusive scans of deg[r] and deg[r] (deg[r] - 1) over r < p by one CTA:
// off[0..p], toff[0..p], cur = off.  Returns the number of terms (thread 0).
__device__ long long cta_scan_rows(const int* deg, int p, int* off, int* toff, int* cur,
                                   long long* s_w) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int chunk = (p + kPolishThreads - 1) / kPolishThreads;
  const int r0 = min(p, t * chunk), r1 = min(p, r0 + chunk);
  long long se = 0, st = 0;
  for (int r = r0; r < r1; ++r) {
    const long long d = __ldcg(deg + r);
    se += d;
    st += d * (d - 1);
  }
  long long ie = se, it = st;  // inclusive scans within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long ye = __shfl_up_sync(FULL, ie, o), yt = __shfl_up_sync(FULL, it, o);
    if (lane >= o) {
      ie += ye;
      it += yt;
    }
  }
  __syncthreads();
  if (lane == 31) {
    s_w[wid] = ie;
    s_w[kWarps + wid] = it;
  }
  __syncthreads();
  long long be = 0, bt = 0;
  for (int k = 0; k < wid; ++k) {
    be += s_w[k];
    bt += s_w[kWarps + k];
  }
  long long e = be + ie - se, tt = bt + it - st;
  for (int r = r0; r < r1; ++r) {
    const long long d = __ldcg(deg + r);
    off[r] = (int)e;
    cur[r] = (int)e;
    toff[r] = tt > 0x7fffffffll ? 0x7fffffff : (int)tt;
    e += d;
    tt += d * (d - 1);
  }
  long long te = 0, tt_all = 0;
  for (int k = 0; k < kWarps; ++k) {
    te += s_w[k];
    tt_all += s_w[kWarps + k];
  }
  if (t == 0) {
    off[p] = (int)te;
    toff[p] = tt_all > 0x7fffffffll ? 0x7fffffff : (int)tt_all;
  }
  return tt_all;
}

// Partial sums of a CTA: warp shuffles, then thread 0 over the warps (fixed
// order), written to partials[blockIdx.x].
__device__ __forceinline__ void block_parts(double (&v)[kParts], double (*s_p)[kParts],
                                            double* partials) {
#pragma unroll
  for (int k = 0; k < kParts; ++k) {
    double x = v[k];
    // skip the tree of warps without terms (tested on the bits); the maxima
    // are of nonnegative values, whose bit patterns order as integers
    const long long xb = __double_as_longlong(x);
    if (__any_sync(FULL, (xb << 1) != 0ll)) {
      if (k == kPartKkt || k == kPartDelta) {
        long long m = xb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
        x = __longlong_as_double(m);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
      }
    }
    v[k] = x;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < kParts; ++k) s_p[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  // the warps' values, part by part, over the lanes of warp 0 (a fixed tree)
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    double* q = partials + (size_t)blockIdx.x * kParts;
#pragma unroll
    for (int k = 0; k < kParts; ++k) {
      double x = lane < kWarps ? s_p[lane][k] : 0.0;  // 0: the identity of both
      if (k == kPartKkt || k == kPartDelta) {
        long long m = __double_as_longlong(x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(FULL, m, o));
        x = __longlong_as_double(m);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
      }
      if (lane == 0) q[k] = x;
    }
  }
}

// The pairs (i, j) of the loud rows i that are not candidates, once each (a
// pair of two loud rows by the smaller row); one warp per (loud row, 32
// columns).  W_ij at the pair's visit takes the entries of row i visited
// before it at their new values and the others (and the diagonal) at their
// old ones; after the sweep all at their new values.  A pair whose Eq. 3
// would leave zero sets the fail flag; a pair beyond the screen's 0.9 lambda
// after the sweep keeps its rows' bounds (loudf 1); the KKT terms are added.
__device__ __forceinline__ void row_sums(const PolishArgs& a, int r, int c, int c_step, int P,
                                         double& at_visit, double& after) {
  const PolishWork& w = a.w;
  const int ld = a.ld;
  const double src = __ldg(a.S + (size_t)r * ld + c);
  double vis = __ldcg(w.diag + r) * src, end = __ldcg(w.diag_new + r) * src;
  const int b = ldi(w.off + r), n = ldi(w.off + r + 1) - b;
  for (int m0 = 0; m0 < n; m0 += 8) {  // loads in batches, then the FMAs in order
    int q[8];
    int2 pr[8];
    double s[8], nv[8], ov[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = m0 + k < n ? ldi(w.ent + b + m0 + k) : -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      pr[k] = q[k] >= 0 ? __ldg(a.cand + q[k]) : make_int2(0, 0);
      nv[k] = q[k] >= 0 ? __ldcg(w.nw + q[k]) : 0.0;
      ov[k] = q[k] >= 0 ? __ldcg(w.om + q[k]) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      s[k] = q[k] >= 0 ? __ldg(a.S + (size_t)other_end(pr[k], r) * ld + c) : 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (q[k] < 0) break;
      vis = ::fma(pair_step(pr[k].x, pr[k].y, P) < c_step ? nv[k] : ov[k], s[k], vis);
      end = ::fma(nv[k], s[k], end);
    }
  }
  at_visit = vis;
  after = end;
}

__device__ __noinline__ void verify_loud(const PolishArgs& a, int nloud, double lam,
                                         double (&v)[kParts], int lane, int swarp, int gwarps,
                                         int P) {
  const PolishWork& w = a.w;
  const int p = a.p;
  const int nchunk = (p + 31) >> 5;
  const double lam_s = (1.0 - kScreenMargin) * lam;
  for (int item = swarp; item < nloud * nchunk; item += gwarps) {
    const int i = ldi(w.loud + item / nchunk);
    const int j = (item % nchunk) * 32 + lane;
    bool pair = j < p && j != i;
    if (pair && j < i && ldi(w.loudf + j) != 0) pair = false;
    {  // candidates are not verified: the row's partners, 32 at a time
      const int b = ldi(w.off + i), n = ldi(w.off + i + 1) - b;
      for (int m0 = 0; m0 < n; m0 += 32) {
        const int mine =
            m0 + lane < n ? other_end(__ldg(a.cand + ldi(w.ent + b + m0 + lane)), i) : -1;
        const int nm = min(32, n - m0);
        for (int m = 0; m < nm; ++m)
          if (__shfl_sync(FULL, mine, m) == j) pair = false;
      }
    }
    if (!pair) continue;
    const int c_step = pair_step(min(i, j), max(i, j), P);
    double vi, ei, vj, ej;
    row_sums(a, i, j, c_step, P, vi, ei);
    row_sums(a, j, i, c_step, P, vj, ej);
    if (soft(-vi - vj, lam) != 0.0) atomicOr(w.ctr + kPolFail, 1);
    const double g = ei + ej;
    if (fabs(g) > lam_s) {
      w.loudf[i] = 1;
      if (ldi(w.loudf + j) != 0) w.loudf[j] = 1;
    }
    v[kPartKkt] = fmax(v[kPartKkt], fmax(fabs(g) - lam, 0.0));
    if (!isfinite(g)) v[kPartBad] += 1.0;
  }
}

__global__ void __launch_bounds__(kPolishThreads, 1) k_polish(const PolishArgs a) {
  const int p = a.p, P = a.P, ld = a.ld;
  const PolishWork& w = a.w;
  const double* __restrict__ S = a.S;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gwarp = gtid >> 5, gwarps = gthreads >> 5;
  // per-candidate and per-row loops run in this order (a permutation of the
  // thread ids): consecutive items go to different CTAs, so the FP64 work of
  // a few thousand candidates spreads over every SM
  const int sid = threadIdx.x * gridDim.x + blockIdx.x;
  const int swarp = wid * (int)gridDim.x + (int)blockIdx.x;  // the same for warps
  const WaitCtl wc = a.wait;
  const double lam = a.lambda;
  unsigned gen = 0;
  int where = 0;
  __shared__ double s_w[2 * kWarps];
  __shared__ double s_p[kWarps][kParts];
  __shared__ int s_steps[kWarps][kSortCap];
  __shared__ double s_res[kRes];
  __shared__ int s_stop;
  const int N = min(__ldg(a.n_cand), w.nc_cap);
  if (threadIdx.x == 0)
    for (int k = 0; k < kRes; ++k) s_res[k] = 0.0;

  // ---- counts per row, the candidates' values, the diagonal, max |s|
  double smax = 0.0;
  for (int k = sid; k < N; k += gthreads) {
    const int2 pr = __ldg(a.cand + k);
    atomicAdd(w.deg + pr.x, 1);
    atomicAdd(w.deg + pr.y, 1);
    w.om[k] = (double)__ldg(a.Om32 + (size_t)pr.x * ld + pr.y);
    w.den[k] = __ldg(a.sdiag + pr.x) + __ldg(a.sdiag + pr.y);
  }
  for (int i = gtid; i < p; i += gthreads) {
    w.diag[i] = __ldg(a.omdiag + i);
    smax = fmax(smax, fmax((double)__ldg(a.mrow + i), fabs(__ldg(a.sdiag + i))));
  }
  {
    const double m = block_max(smax, s_w);
    if (threadIdx.x == 0) atomic_max_nonneg(w.ctr + kPolSMax, m);
  }
  grid_barrier(a.barrier, gen, wc, ++where);
  // ---- row offsets of the entries and the terms (one CTA)
  if (blockIdx.x == 0) {
    const long long terms = cta_scan_rows(w.deg, p, w.off, w.toff, w.cur,
                                          reinterpret_cast<long long*>(s_w));
    if (threadIdx.x == 0 && terms > (long long)w.term_cap)
      w.ctr[kPolOverflow] = terms > 0x7fffffffll ? 0x7fffffff : (int)terms;
  }
  grid_barrier(a.barrier, gen, wc, ++where);
  int status = 1;  // not converged (the sweep budget ran out)
  int sweeps = 0;
  const bool overflow = ldi(w.ctr + kPolOverflow) != 0;
  if (overflow) status = kStatusCapacity;
  if (!overflow) {
    // ---- row entries (in any order), then ranked by colour step
    for (int k = sid; k < N; k += gthreads) {
      const int2 pr = __ldg(a.cand + k);
      w.ent0[atomicAdd(w.cur + pr.x, 1)] = k;
      w.ent0[atomicAdd(w.cur + pr.y, 1)] = k;
    }
    grid_barrier(a.barrier, gen, wc, ++where);
    for (int r = gwarp; r < p; r += gwarps) {
      const int b = ldi(w.off + r), n = ldi(w.off + r + 1) - b;
      const bool staged = n <= kSortCap;
      if (staged)
        for (int m = lane; m < n; m += 32) {
          const int2 pr = __ldg(a.cand + ldi(w.ent0 + b + m));
          s_steps[wid][m] = pair_step(pr.x, pr.y, P);
        }
      __syncwarp();
      double rs = 0.0;
      for (int m = lane; m < n; m += 32) {
        const int q = ldi(w.ent0 + b + m);
        const int2 pr = __ldg(a.cand + q);
        const int st = staged ? s_steps[wid][m] : pair_step(pr.x, pr.y, P);
        int rank = 0;
        for (int m2 = 0; m2 < n; ++m2) {
          int st2;
          if (staged) {
            st2 = s_steps[wid][m2];
          } else {
            const int2 p2 = __ldg(a.cand + ldi(w.ent0 + b + m2));
            st2 = pair_step(p2.x, p2.y, P);
          }
          rank += st2 < st ? 1 : 0;  // the steps of a row are distinct
        }
        w.ent[b + rank] = q;
        w.pos[2 * q + (pr.x == r ? 0 : 1)] = rank;
        rs += fabs(__ldcg(w.om + q));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(FULL, rs, o);
      __syncwarp();
    }
    grid_barrier(a.barrier, gen, wc, ++where);
    // ---- terms of each (candidate, side): the other entries of the row, in
    //      colour-step order (the first pos of them precede the candidate),
    //      with the S entry each multiplies in the candidate's sum
    for (int x = sid; x < 2 * N; x += gthreads) {
      const int k = x >> 1, sd = x & 1;
      const int2 pr = __ldg(a.cand + k);
      const int r = sd ? pr.y : pr.x, c = sd ? pr.x : pr.y;
      const int b = ldi(w.off + r), n = ldi(w.off + r + 1) - b;
      const int self = ldi(w.pos + x);
      const size_t t0 = (size_t)ldi(w.toff + r) + (size_t)self * (n - 1);
      int t = 0;
      for (int m = 0; m < n; ++m) {
        if (m == self) continue;
        const int q = ldi(w.ent + b + m);
        const int u = other_end(__ldg(a.cand + q), r);
        w.term_q[t0 + t] = q;
        w.term_s[t0 + t] = __ldg(S + (size_t)u * ld + c);
        ++t;
      }
    }
    // per-row bound carried from the FP32 phase, plus the change of S under
    // the iterate: |G_ij(S64) - G_ij(S32)| <= (||Omega_i||_1 + ||Omega_j||_1)
    // max|dS|, with max|dS| the refined entries' largest change or FP32
    // rounding of S
    {
      const double ds_ref = a.ds_bits ? (double)__int_as_float(__ldg(a.ds_bits)) : 0.0;
      const double ds = fmax(ds_ref, ld_nonneg(w.ctr + kPolSMax) * 0x1p-24);
      for (int r = sid; r < p; r += gthreads) {
        const int b = ldi(w.off + r), n = ldi(w.off + r + 1) - b;
        double rs = fabs(__ldcg(w.diag + r));
        for (int m = 0; m < n; ++m) rs += fabs(__ldcg(w.om + ldi(w.ent + b + m)));
        w.rowa[r] = (a.rowacc ? __ldcg(a.rowacc + r) : 0.5 * a.acc0) + rs * ds;
      }
    }
    grid_barrier(a.barrier, gen, wc, ++where);
    const double half_bound = 0.5 * (kScreenMargin - kLazySlack) * lam;
    int gr = 0;  // fixed-point rounds so far (all sweeps): selects the flag slot
    int first_delta = 0;
  int n_partial = 0;  // sweeps that verified loud rows
    for (int t = 0; t < a.n_sweeps; ++t) {
      // ---- base sums at the sweep's start (fixed order: diagonal, then the
      //      row's other entries in colour-step order)
      if (gtid == 0) {
        w.ctr[kPolLoud] = 0;
        w.ctr[kPolFail] = 0;
      }
      for (int x = sid; x < 2 * N; x += gthreads) {
        const int k = x >> 1, sd = x & 1;
        const int2 pr = __ldg(a.cand + k);
        const int r = sd ? pr.y : pr.x, c = sd ? pr.x : pr.y;
        const int n = ldi(w.off + r + 1) - ldi(w.off + r);
        const size_t t0 = (size_t)ldi(w.toff + r) + (size_t)ldi(w.pos + x) * (n - 1);
        double s = __ldcg(w.diag + r) * __ldg(S + (size_t)r * ld + c);
        for (int m = 0; m < n - 1; ++m)
          s = ::fma(__ldcg(w.om + ldi(w.term_q + t0 + m)), __ldcg(w.term_s + t0 + m), s);
        w.base[x] = s;
        if (!sd) w.d0[k] = 0.0;
      }
      grid_barrier(a.barrier, gen, wc, ++where);
      // ---- the chain: fixed-point rounds of Eq. 3 over the candidates.
      //      The thread's first candidate keeps what the rounds reuse in
      //      registers (its sums at the sweep start, its denominator, value,
      //      and the first kQ terms of each side), so a round waits on one
      //      level of loads: the earlier candidates' current changes
      double* dc = w.d0;
      double* dn = w.d1;
      bool settled = false;
      const int k0 = sid;
      double c_a1 = 0.0, c_a2 = 0.0, c_den = 1.0, c_om = 0.0, c_d = 0.0;
      int c_pi = 0, c_pj = 0;
      size_t c_ti = 0, c_tj = 0;
      int c_qi[kQ], c_qj[kQ];
      double c_si[kQ], c_sj[kQ];
      if (k0 < N) {
        const int2 pr = __ldg(a.cand + k0);
        const int ni = ldi(w.off + pr.x + 1) - ldi(w.off + pr.x);
        const int nj = ldi(w.off + pr.y + 1) - ldi(w.off + pr.y);
        c_pi = ldi(w.pos + 2 * k0);
        c_pj = ldi(w.pos + 2 * k0 + 1);
        c_ti = (size_t)ldi(w.toff + pr.x) + (size_t)c_pi * (ni - 1);
        c_tj = (size_t)ldi(w.toff + pr.y) + (size_t)c_pj * (nj - 1);
        c_a1 = __ldcg(w.base + 2 * k0);
        c_a2 = __ldcg(w.base + 2 * k0 + 1);
        c_den = __ldcg(w.den + k0);
        c_om = __ldcg(w.om + k0);
      }
#pragma unroll
      for (int m = 0; m < kQ; ++m) {
        c_qi[m] = m < c_pi ? ldi(w.term_q + c_ti + m) : 0;
        c_si[m] = m < c_pi ? __ldcg(w.term_s + c_ti + m) : 0.0;
        c_qj[m] = m < c_pj ? ldi(w.term_q + c_tj + m) : 0;
        c_sj[m] = m < c_pj ? __ldcg(w.term_s + c_tj + m) : 0.0;
      }
      for (int rnd = 0; rnd < kPolishMaxRounds; ++rnd, ++gr) {
        if (gtid == 0) w.rslot[(gr + 1) % 3] = 0ull;  // waited on two rounds ago
        bool chg = false;
        if (k0 < N) {
          double x1[kQ], x2[kQ];
#pragma unroll
          for (int m = 0; m < kQ; ++m) {  // issued together, then summed in order
            x1[m] = m < c_pi ? __ldcg(dc + c_qi[m]) : 0.0;
            x2[m] = m < c_pj ? __ldcg(dc + c_qj[m]) : 0.0;
          }
          double a1 = c_a1, a2 = c_a2;
#pragma unroll
          for (int m = 0; m < kQ; ++m) {
            if (m < c_pi) a1 = ::fma(x1[m], c_si[m], a1);
            if (m < c_pj) a2 = ::fma(x2[m], c_sj[m], a2);
          }
          for (int m = kQ; m < c_pi; ++m)
            a1 = ::fma(__ldcg(dc + ldi(w.term_q + c_ti + m)), __ldcg(w.term_s + c_ti + m), a1);
          for (int m = kQ; m < c_pj; ++m)
            a2 = ::fma(__ldcg(dc + ldi(w.term_q + c_tj + m)), __ldcg(w.term_s + c_tj + m), a2);
          const double nv = soft(-a1 - a2, lam) / c_den;
          const double d = nv - c_om;
          chg |= __double_as_longlong(d) != __double_as_longlong(c_d);
          c_d = d;
          dn[k0] = d;
          w.nw[k0] = nv;
        }
        for (int k = sid + gthreads; k < N; k += gthreads) {
          const int2 pr = __ldg(a.cand + k);
          const int ni = ldi(w.off + pr.x + 1) - ldi(w.off + pr.x);
          const int nj = ldi(w.off + pr.y + 1) - ldi(w.off + pr.y);
          const int pi = ldi(w.pos + 2 * k), pj = ldi(w.pos + 2 * k + 1);
          const size_t ti = (size_t)ldi(w.toff + pr.x) + (size_t)pi * (ni - 1);
          const size_t tj = (size_t)ldi(w.toff + pr.y) + (size_t)pj * (nj - 1);
          double a1 = __ldcg(w.base + 2 * k), a2 = __ldcg(w.base + 2 * k + 1);
          for (int m = 0; m < pi; ++m)
            a1 = ::fma(__ldcg(dc + ldi(w.term_q + ti + m)), __ldcg(w.term_s + ti + m), a1);
          for (int m = 0; m < pj; ++m)
            a2 = ::fma(__ldcg(dc + ldi(w.term_q + tj + m)), __ldcg(w.term_s + tj + m), a2);
          const double nv = soft(-a1 - a2, lam) / __ldcg(w.den + k);
          const double d = nv - __ldcg(w.om + k);
          chg |= __double_as_longlong(d) != __double_as_longlong(__ldcg(dc + k));
          dn[k] = d;
          w.nw[k] = nv;
        }
        const bool moved = round_barrier_any(w.rslot + gr % 3, gridDim.x, chg, wc, ++where,
                                             (int)blockIdx.x);
        double* tmp = dc;
        dc = dn;
        dn = tmp;
        if (!moved) {
          settled = true;
          ++gr;
          break;
        }
        if (ld_relaxed_s32(wc.abort) != 0) break;
      }
      if (ld_relaxed_s32(wc.abort) != 0) {
        status = 3;
        break;
      }
      if (!settled) {
        status = kStatusNeedW;
        break;
      }
      // ---- diagonal (Eq. 2) with the new off-diagonal values; row bounds;
      //      the diagonal's objective / KKT terms
      double v[kParts];
#pragma unroll
      for (int k = 0; k < kParts; ++k) v[k] = 0.0;
      for (int r = sid; r < p; r += gthreads) {
        const int b = ldi(w.off + r), n = ldi(w.off + r + 1) - b;
        double cr = 0.0, dsum = 0.0;
        for (int m = 0; m < n; ++m) {
          const int q = ldi(w.ent + b + m);
          const int u = other_end(__ldg(a.cand + q), r);
          cr = ::fma(__ldcg(w.nw + q), __ldg(S + (size_t)u * ld + r), cr);
          dsum += fabs(__ldcg(dc + q)) * (double)__ldg(a.mrow + u);
        }
        const double sii = __ldg(a.sdiag + r), oii = __ldcg(w.diag + r);
        const double nd = (-cr + sqrt(cr * cr + 4.0 * sii)) / (2.0 * sii);
        const double dw = nd - oii;
        w.diag_new[r] = nd;
        const double rb = __ldcg(w.rowa + r) + dsum + fabs(dw) * (double)__ldg(a.mrow + r);
        w.rowb[r] = rb;
        const bool loud = !(rb <= half_bound);
        w.loudf[r] = loud ? 2 : 0;  // 2: loud, its pairs within 0.9 lambda so far
        if (loud) {
          const int slot = atomicAdd(w.ctr + kPolLoud, 1);
          if (slot < kPolLoudMax) w.loud[slot] = r;
        }
        const double wd = ::fma(nd, sii, cr);  // W_rr after the sweep
        v[kPartDelta] = fmax(v[kPartDelta], fabs(dw));
        if (nd > 0.0 && isfinite(wd) && isfinite(nd)) {
          v[kPartKkt] = fmax(v[kPartKkt], fabs(wd - 1.0 / nd));
          v[kPartQuad] += nd * wd;
          v[kPartLog] += log(nd);
        } else {
          v[kPartBad] += 1.0;
        }
      }
      grid_barrier(a.barrier, gen, wc, ++where);
      // ---- decision (every CTA alike).  A pair outside the list has moved
      //      by at most rowb_i + rowb_j since it was screened: pairs of two
      //      rows within half the margin stay at zero.  The pairs of the
      //      other rows (a few) are verified exactly: Eq. 3's zero test at
      //      their visit, from the sums over the nonzeros of rows i and j
      //      with the values each had at that step.  Too many such rows, or
      //      a pair that would have left zero: nothing of this sweep is
      //      committed (W is rebuilt and the screened polish takes over)
      const int nloud = ldi(w.ctr + kPolLoud);
      if (nloud > kPolLoudMax) {
        status = kStatusNeedW;
        break;
      }
      if (nloud > 0) {
        ++n_partial;
        verify_loud(a, nloud, lam, v, lane, swarp, gwarps, P);
        grid_barrier(a.barrier, gen, wc, ++where);
        if (ldi(w.ctr + kPolFail) != 0) {
          status = kStatusNeedW;
          break;
        }
      }
      // ---- commit
      for (int k = sid; k < N; k += gthreads) {
        const double d = __ldcg(dc + k);
        if (d != 0.0) {
          w.om[k] = __ldcg(w.nw + k);
          v[kPartDelta] = fmax(v[kPartDelta], fabs(d));
          v[kPartActive] += 2.0;
        }
      }
      for (int r = sid; r < p; r += gthreads) {
        w.diag[r] = __ldcg(w.diag_new + r);
        // a verified row whose pairs all stayed within 0.9 lambda restarts
        // its bound; every other row keeps its bound, grown by the sweep
        w.rowa[r] = ldi(w.loudf + r) == 2 ? 0.0 : __ldcg(w.rowb + r);
      }
      grid_barrier(a.barrier, gen, wc, ++where);
      // ---- the candidates' objective / KKT terms after the sweep:
      //      W_ij = omega_ii s_ij + sum_{u in N(i), u != j} omega_iu s_uj +
      //      omega_ij s_jj (and W_ji alike), G = W_ij + W_ji
      for (int k = sid; k < N; k += gthreads) {
        const int2 pr = __ldg(a.cand + k);
        const double om = __ldcg(w.om + k);
        double g = 0.0;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int r = sd ? pr.y : pr.x, c = sd ? pr.x : pr.y;
          const int n = ldi(w.off + r + 1) - ldi(w.off + r);
          const size_t t0 = (size_t)ldi(w.toff + r) + (size_t)ldi(w.pos + 2 * k + sd) * (n - 1);
          double s = __ldcg(w.diag + r) * __ldg(S + (size_t)r * ld + c);
          for (int m = 0; m < n - 1; ++m)
            s = ::fma(__ldcg(w.om + ldi(w.term_q + t0 + m)), __ldcg(w.term_s + t0 + m), s);
          s = ::fma(om, __ldg(a.sdiag + c), s);
          g += s;
        }
        v[kPartKkt] = fmax(v[kPartKkt], kkt_offdiag(om, g, lam));
        v[kPartQuad] += om * g;
        v[kPartPen] += fabs(om);
        if (!isfinite(g) || !isfinite(om)) v[kPartBad] += 1.0;
      }
      block_parts(v, s_p, a.partials);
      grid_barrier(a.barrier, gen, wc, ++where);
      // ---- every CTA reduces the partials identically (warp 0: lanes stride
      //      over the CTAs, then a fixed shuffle tree)
      double kkt = 0.0, quad = 0.0, pen = 0.0, lg = 0.0, dl = 0.0, ac = 0.0, bad = 0.0;
      if (wid == 0) {
        for (int c = lane; c < (int)gridDim.x; c += 32) {
          const double* q = a.partials + (size_t)c * kParts;
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
      sweeps = t + 1;
      if (threadIdx.x == 0) {
        const double obj = -lg + 0.5 * quad + lam * pen;
        const bool aborted = ld_relaxed_s32(wc.abort) != 0;
        const bool nonfinite = bad > 0.0 || !isfinite(obj) || !isfinite(kkt);
        if (first_delta == 0 && dl < a.delta_tol) first_delta = sweeps;
        const bool conv = (a.stop_rule == 1) ? (dl < a.tol) : (kkt <= a.tol);
        s_res[kResKkt] = kkt;
        s_res[kResObj] = obj;
        s_res[kResDelta] = dl;
        s_res[kResActive] = ac * 0.5;
        const int code = aborted ? 3 : nonfinite ? 2 : conv ? 0 : 1;
        s_res[kResStatus] = code;
        s_stop = (code != 1 || sweeps >= a.n_sweeps) ? 1 : 0;
        if (blockIdx.x == 0 && t < a.hist_len) {
          double* h = a.hist + (size_t)t * kHist;
          h[0] = dl;
          h[1] = kkt;
          h[2] = obj;
          h[3] = ac * 0.5;
        }
      }
      __syncthreads();
      status = (int)s_res[kResStatus];
      if (s_stop) break;
    }
    if (threadIdx.x == 0) {
      s_res[kResFirstDelta] = first_delta;
      s_res[kResAcc] = 0.0;
      s_res[kResPartial] = n_partial;
    }
  }
  // ---- the iterate into the zeroed FP64 Omega (both triangles; every
  //      nonzero off the diagonal is a candidate), also when the terms did
  //      not fit (the values loaded at the start)
  for (int k = sid; k < N; k += gthreads) {
    const int2 pr = __ldg(a.cand + k);
    const double om = __ldcg(w.om + k);
    a.Om[(size_t)pr.x * ld + pr.y] = om;
    a.Om[(size_t)pr.y * ld + pr.x] = om;
  }
  for (int r = gtid; r < p; r += gthreads) a.Om[(size_t)r * ld + r] = __ldcg(w.diag + r);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s_res[kResSweeps] = sweeps;
    s_res[kResStatus] = status;
    s_res[kResRedo] = 0.0;
    s_res[kResPath] = 0.0;
    s_res[kResList] = -1.0;
    s_res[kResLazy] = sweeps;
    for (int k = 0; k < kRes; ++k) a.result[k] = s_res[k];
  }
}

}  // namespace

cudaError_t launch_polish(const PolishArgs& a, int grid, cudaStream_t st) {
  note_launches(1);
  void* kargs[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)k_polish, dim3(grid), dim3(kPolishThreads), kargs,
                                     0, st);
}

}  // namespace concord
