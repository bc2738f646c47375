// CONCORD-PCD sweep: one persistent cooperative kernel per call that runs
// Algorithm 1's outer iterations (all colour steps, then the diagonal step)
// and the fused objective / KKT / delta reduction after every sweep.
//
// Work decomposition (GB300-first, not the paper's kernel design):
//   * Warp w owns rows {w, w + TW, w + 2 TW, ...} (TW = warps in the grid):
//     Omega row i, W row i = (Omega S)_i.  Lane k of the warp carries the
//     scalar work of the k-th owned row.
//   * Colour step c pairs row i with j = partner(i, c) (closed-form circle
//     method).  The update of Eq. 3 needs W_ij (row i, local) and W_ji (row j,
//     owned elsewhere): the two owners swap exactly these scalars through an
//     L2-resident mailbox ring, then both compute the identical new value in
//     the canonical (min, max) order, so Omega stays exactly symmetric
//     (Lemma 1: nothing else of the colour's other pairs is read).
//   * If the value moved by delta, each owner updates its own W row:
//     W_i += delta S_j (W_j += delta S_i on the other side).  The next step's
//     published scalar is formed first with the same FMA, so the row update
//     overlaps the partner exchange.
//   * No grid-wide barrier inside a sweep: a row advances as soon as its
//     partner has published.  One grid barrier per sweep precedes the fused
//     KKT / objective pass; a second one publishes its partial results.
#include "common.cuh"
#include "kernels.h"

namespace concord {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
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
struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void fma(V& w, double d, const V& s) {
    w.x = ::fma(d, s.x, w.x);
    w.y = ::fma(d, s.y, w.y);
  }
};

__device__ __forceinline__ float fma_t(float d, float s, float w) { return fmaf(d, s, w); }
__device__ __forceinline__ double fma_t(double d, double s, double w) { return ::fma(d, s, w); }

// W_row += d * S_row over the padded width ld (a multiple of 32 elements; the
// padding of S is zero, so the padding of W stays zero).  16-byte vectors,
// lanes interleaved so each warp instruction touches 512 contiguous bytes.
template <typename T>
__device__ __forceinline__ void axpy_row(T* __restrict__ w, const T* __restrict__ s, T d, int ld,
                                         int lane) {
  using VT = Vec16<T>;
  using V = typename VT::V;
  const int nv = ld / VT::N;
  V* wv = reinterpret_cast<V*>(w);
  const V* sv = reinterpret_cast<const V*>(s);
  int k = lane;
  for (; k + 96 < nv; k += 128) {
    V s0 = __ldg(sv + k), s1 = __ldg(sv + k + 32), s2 = __ldg(sv + k + 64), s3 = __ldg(sv + k + 96);
    V w0 = wv[k], w1 = wv[k + 32], w2 = wv[k + 64], w3 = wv[k + 96];
    VT::fma(w0, d, s0);
    VT::fma(w1, d, s1);
    VT::fma(w2, d, s2);
    VT::fma(w3, d, s3);
    wv[k] = w0;
    wv[k + 32] = w1;
    wv[k + 64] = w2;
    wv[k + 96] = w3;
  }
  for (; k < nv; k += 32) {
    V s0 = __ldg(sv + k);
    V w0 = wv[k];
    VT::fma(w0, d, s0);
    wv[k] = w0;
  }
}

template <typename T>
__device__ __forceinline__ T soft_threshold(T x, T tau) {
  T a = fabs(x) - tau;
  if (!(a > (T)0)) return (T)0;
  return x > (T)0 ? a : -a;
}

// Block reduction of the per-thread partials into partials[blockIdx.x*kParts+k].
__device__ __forceinline__ void block_reduce_parts(double (&v)[kParts], double* out,
                                                   double (*red)[kParts], int slot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < kParts; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_down_sync(0xffffffffu, x, o);
      x = (k == kPartKkt || k == kPartDelta) ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[wid][k] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < kParts; ++k) {
      double x = red[0][k];
      for (int w = 1; w < nw; ++w)
        x = (k == kPartKkt || k == kPartDelta) ? fmax(x, red[w][k]) : x + red[w][k];
      out[(size_t)slot * kParts + k] = x;
    }
  }
  __syncthreads();
}

// Partner of row v at the colour whose ring index is r (rows v >= 1): the
// closed form of cm_partner with the ring index kept incrementally.
__device__ __forceinline__ int ring_partner(int r, int v) { return (r + 1 == v) ? 0 : r + 1; }
__device__ __forceinline__ int ring_norm(int r, int P) {
  while (r < 0) r += P;
  while (r >= P) r -= P;
  return r;
}

__device__ __forceinline__ void prefetch_l1(const void* ptr) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr));
}

// Apply a row's pending updates in order: W_row[x] <- fma(d_k, S[u_k][x], .)
// for k = 0..cnt-1, for every x of the padded row (the same FMA chain the
// eager row updates would have applied one at a time).  The whole warp
// cooperates; pu / pd are the row's pending columns / changes (stride `st`).
template <typename T>
__device__ __forceinline__ void flush_row(T* __restrict__ w, const T* __restrict__ S, const int* pu,
                                          const T* pd, int st, int cnt, int ld, int lane) {
  using VT = Vec16<T>;
  using V = typename VT::V;
  const int nv = ld / VT::N;
  V* wv = reinterpret_cast<V*>(w);
  for (int k0 = lane; k0 < nv; k0 += 64) {
    const bool two = k0 + 32 < nv;
    V a = wv[k0];
    V b = two ? wv[k0 + 32] : a;
    for (int k = 0; k < cnt; ++k) {
      const V* sv = reinterpret_cast<const V*>(S + (size_t)pu[k * st] * ld);
      const T d = pd[k * st];
      V sa = __ldg(sv + k0);
      V sb = two ? __ldg(sv + k0 + 32) : sa;
      VT::fma(a, d, sa);
      VT::fma(b, d, sb);
    }
    wv[k0] = a;
    if (two) wv[k0 + 32] = b;
  }
}

// DSMEM helpers (cluster variant): stores into / loads from the shared
// memory of another CTA of the cluster through its generic address.
__device__ __forceinline__ void st_cluster_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.cluster.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v2u64(unsigned long long* p, unsigned long long a,
                                                 unsigned long long b) {
  asm volatile("st.relaxed.cluster.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned ld_cluster_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_cluster_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.cluster.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void* map_rank(void* p, unsigned rank) {
  unsigned long long out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return (void*)out;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Cluster mailbox word of a 32- or 64-bit value: (tag << 32 | bits) words.
template <typename T>
__device__ __forceinline__ void box_store(unsigned long long* remote, unsigned tag, T v);
template <>
__device__ __forceinline__ void box_store<float>(unsigned long long* remote, unsigned tag, float v) {
  st_cluster_u64(remote, ((unsigned long long)tag << 32) | __float_as_uint(v));
}
template <>
__device__ __forceinline__ void box_store<double>(unsigned long long* remote, unsigned tag, double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long t = (unsigned long long)tag << 32;
  st_cluster_v2u64(remote, t | (b >> 32), t | (b & 0xffffffffull));
}
template <typename T>
__device__ __forceinline__ bool box_read(const unsigned long long* local, unsigned tag, T& v);
template <>
__device__ __forceinline__ bool box_read<float>(const unsigned long long* local, unsigned tag, float& v) {
  const unsigned long long w = ld_cluster_u64(local);
  v = __uint_as_float((unsigned)(w & 0xffffffffull));
  return (unsigned)(w >> 32) == tag;
}
template <>
__device__ __forceinline__ bool box_read<double>(const unsigned long long* local, unsigned tag, double& v) {
  const unsigned long long hi = ld_cluster_u64(local), lo = ld_cluster_u64(local + 1);
  v = __longlong_as_double((long long)(((hi & 0xffffffffull) << 32) | (lo & 0xffffffffull)));
  return (unsigned)(hi >> 32) == tag && (unsigned)(lo >> 32) == tag;
}

// One persistent launch of Algorithm 1's outer iterations.
//   CLUSTER = false: persistent cooperative grid (one CTA per SM); the two
//     owners of a pair swap their W scalars through an L2 mailbox ring.
//   CLUSTER = true: the whole grid is one thread-block cluster; the mailbox
//     word a row reads lives in its own CTA's shared memory and the partner
//     stores into it through distributed shared memory (lower latency), with
//     per-row progress counters guarding slot reuse.
//   BATCH = true (grid form): the launch serves a.n_probs independent
//     problems; each CTA belongs to one problem (its CTA range), whose rows,
//     mailbox ring, barriers and partial sums are its own, and each problem
//     walks the lambda path a.lambdas (warm-started) at its own pace.
template <typename T>
__device__ __forceinline__ const SweepArgs<T>& pick_args(const SweepArgs<T>& batch,
                                                          const SweepArgs<T>& single,
                                                          bool use_batch) {
  return use_batch ? batch : single;
}

template <typename T, bool MIXED, bool CLUSTER, bool BATCH>
__global__ void __launch_bounds__(kSweepThreads, 1) k_sweep(const SweepArgs<T> a) {
  using MB = Mailbox<T>;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int KC = kPendCap;
  constexpr int BW = sizeof(T) / 4;  // cluster mailbox words per value
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  // The CTA's problem: the launch's own arguments, or (batch) a copy with the
  // problem's dimension, arrays and counters; G / cta are the CTA count and
  // index within the problem's group.
  __shared__ SweepArgs<T> s_args;
  __shared__ int s_gc[2];
  int G = gridDim.x, cta = blockIdx.x;
  if constexpr (BATCH) {
    if (threadIdx.x == 0) {
      int lo = 0, hi = a.n_probs - 1;
      while (lo < hi) {  // last problem whose range starts at or before this CTA
        const int mid = (lo + hi + 1) >> 1;
        if (a.probs[mid].cta0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
      }
      const BatchProblem<T>& q = a.probs[lo];
      s_args = a;
      s_args.p = q.p;
      s_args.P = q.P;
      s_args.ld = q.ld;
      s_args.W = q.W;
      s_args.Om = q.Om;
      s_args.S = q.S;
      s_args.sdiag = q.sdiag;
      s_args.sd1 = q.sd1;
      s_args.sd2 = q.sd2;
      s_args.sdiag64 = q.sdiag64;
      s_args.omdiag64 = q.omdiag64;
      s_args.mbox = q.mbox;
      s_args.barrier = q.barrier;
      s_args.partials = q.partials;
      s_args.result = q.result;
      s_args.batch_cnt = q.cnt;
      s_args.stall_break = q.stall_break;
      if (q.n_sweeps > 0) s_args.n_sweeps = q.n_sweeps;
      s_args.lambdas = a.lambdas + q.k0;
      s_args.n_lambda = q.nk;
      s_args.hist_len = 0;
      s_args.fault_vertex = -1;
      s_args.fault_step = -1;
      s_args.lambda = a.lambdas[q.k0];
      s_gc[0] = q.ctas;
      s_gc[1] = (int)blockIdx.x - q.cta0;
    }
    __syncthreads();
    G = s_gc[0];
    cta = s_gc[1];
  }
  const SweepArgs<T>& A = pick_args<T>(s_args, a, BATCH);
  const bool row_warp = wid < A.row_warps;
  const int p = A.p, P = A.P, ld = A.ld;
  const int pe = P + 1;
  const int R = A.rows_per_warp;
  const int CS = G;                   // cluster: CTAs in the cluster (a power of two)
  const int cs_log2 = __ffs(CS) - 1;
  const int cap = A.row_warps * R;            // cluster: rows a CTA can hold
  const int li = wid * R + lane;              // cluster: local index of this lane's row
  int myrow;
  if constexpr (CLUSTER) {
    myrow = li * CS + (int)cta;
  } else {
    myrow = (cta * A.row_warps + wid) + lane * (G * A.row_warps);
  }
  const bool has_row = row_warp && lane < R && myrow < p;
  // the lambda in force (batch: walks the path, index kl)
  double lam_cur = A.lambda;
  T lam = (T)lam_cur;
  int kl = 0;
  const WaitCtl& wc = A.wait;

  __shared__ double red[kSweepThreads / 32][kParts];
  __shared__ int s_stop, s_lam_end, s_lam_count;
  __shared__ double s_res[kRes];
  // Dynamic shared memory: pending (not yet applied) row updates of every
  // owned row -- entry k of lane l of row warp w at ((w * KC + k) * R + l) --
  // then, for the cluster variant, the mailbox ring box[kDepth][cap][BW] and
  // the per-row progress counters prog[cap].
  extern __shared__ __align__(16) unsigned char dyn[];
  T* pd_all = reinterpret_cast<T*>(dyn);
  int* pu_all = reinterpret_cast<int*>(dyn + sizeof(T) * (size_t)A.row_warps * KC * R);
  unsigned long long* box = reinterpret_cast<unsigned long long*>(
      dyn + (sizeof(T) + sizeof(int)) * (size_t)A.row_warps * KC * R);
  unsigned* prog = reinterpret_cast<unsigned*>(box + (size_t)kDepth * cap * BW);
  const int pst = R;
  T* pd = pd_all + (size_t)(row_warp ? wid : 0) * KC * R + (lane < R ? lane : 0);
  int* pu = pu_all + (size_t)(row_warp ? wid : 0) * KC * R + (lane < R ? lane : 0);

  // cluster: step tags restart at 1 every launch (fresh shared memory)
  const unsigned tag_base = CLUSTER ? 1u : A.tag_base;
  if constexpr (CLUSTER) {
    for (int e = threadIdx.x; e < kDepth * cap * BW; e += blockDim.x) box[e] = 0ull;
    for (int e = threadIdx.x; e < cap; e += blockDim.x) prog[e] = 0u;
    cluster_sync_all();
  }

  unsigned gen = 0;
  int first_delta = 0;
  double best_kkt = 1e300;
  int since_best = 0;
  int t = 0;      // sweeps of this launch (mailbox tags)
  int t_lam = 0;  // batch: sweeps at the current lambda
  T* __restrict__ Wrow = A.W + (size_t)(has_row ? myrow : 0) * ld;
  T* __restrict__ Orow = A.Om + (size_t)(has_row ? myrow : 0) * ld;
  const T s_mine = has_row ? A.sdiag[myrow] : (T)1;

  for (;;) {
    const bool do_sweep = !A.kkt_only && (BATCH ? t_lam : t) < A.n_sweeps;
    double dmax = 0.0, nact = 0.0;
    if (do_sweep && row_warp) {
      const unsigned step0 = tag_base + (unsigned)(t * P);
      int cnt = 0;  // pending updates of this lane's row
      // Partners without integer division: for v >= 1 the ring index
      // (-v - 1 - 2c) mod P drops by 2 per colour; vertex 0 meets P - c.
      int j = has_row ? cm_partner(myrow, 0, P) : p;
      int rr = 0;  // ring index of colour c + 1 (rows v >= 1)
      if (has_row && myrow > 0) {
        rr = (-myrow - 3) % P;
        if (rr < 0) rr += P;
      }
      // j1: partner at colour 1 (the next step's partner during step 0)
      int j1 = p;
      if (has_row && P > 1) j1 = (myrow == 0) ? (P - 1) : ((rr + 1 == myrow) ? 0 : rr + 1);
      T pub = (has_row && j < p) ? Wrow[j] : (T)0;
      // Operands of the current step, loaded one step ahead (register
      // pipeline): om / so = w_ij and s_jj of this step's pair; sjn =
      // S[j][j_next]; wA = W_i,j_next with the pending updates counted in nA
      // still to be added (their S values gathered into g[]), plus dprev *
      // sprev for the update made one step earlier.
      T om = (T)0, so = (T)1, sjn = (T)0, wA = (T)0, sprev = (T)0, dprev = (T)0;
      T g[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) g[k] = (T)0;
      int nA = 0;
      if (has_row && j < p) {
        om = Orow[j];
        so = A.sdiag[j];
        if (j1 < p) {
          if (myrow == 0)
            sjn = A.sd1[j];
          else if (j != 0 && j1 != 0)
            sjn = A.sd2[j];
          else
            sjn = __ldg(A.S + (size_t)j * ld + j1);
        }
      }
      if (has_row && j1 < p) wA = Wrow[j1];
      // Step 0 of a sweep reuses a slot whose reader finished the previous
      // sweep (barrier) or launch: no check needed.
      if (has_row && !(myrow == A.fault_vertex && t * P == A.fault_step)) {
        if constexpr (CLUSTER) {
          if (j < p)
            box_store<T>((unsigned long long*)map_rank(
                             box + ((size_t)(step0 & (kDepth - 1)) * cap + (j >> cs_log2)) * BW, j & (CS - 1)),
                         step0, pub);
        } else {
          MB::publish(A.mbox + ((size_t)(step0 & (kDepth - 1)) * pe + myrow) * MB::kWords, step0,
                      pub);
        }
      }
      int jn = j1;  // partner of step c + 1
      // slot-reuse guards in flight (see the loop): for iteration c + 1 and c + 2
      const unsigned long long *rw_next = nullptr, *rw_new = nullptr;
      const unsigned *rp_next = nullptr, *rp_new = nullptr;
      unsigned rtag_next = 0xffffffffu, rtag_new = 0xffffffffu;
      for (int c = 0; c < P; ++c) {
        const unsigned step = step0 + (unsigned)c;
        const int slot = (int)(step & (kDepth - 1));
        const bool paired = has_row && j < p;
        const bool more = c + 1 < P;
        // -- the partner's W_ji: issue its load first
        T wji = (T)0;
        const unsigned long long* src;
        if constexpr (CLUSTER)
          src = box + ((size_t)slot * cap + (li < cap ? li : 0)) * BW;
        else
          src = A.mbox + ((size_t)slot * pe + (paired ? j : 0)) * MB::kWords;
        bool done;
        if constexpr (CLUSTER)
          done = !paired || box_read<T>(src, step, wji);
        else
          done = !paired || MB::try_read(src, step, wji);
        // -- partner of step c + 2 and the next step's scalar operands
        int jnn = p;
        if (has_row && c + 2 < P) {
          int r2 = rr - 2;
          while (r2 < 0) r2 += P;
          jnn = (myrow == 0) ? (P - (c + 2)) : ((r2 + 1 == myrow) ? 0 : r2 + 1);
        }
        T om_n = (T)0, so_n = (T)1, sjn_n = (T)0;
        if (has_row && jn < p) {
          om_n = Orow[jn];
          so_n = A.sdiag[jn];
          // S[j_(c+1)][j_(c+2)]: consecutive partners are neighbours on the
          // cyclic ring (second sub-diagonal; the first for row 0) except
          // around vertex 0, so this is a walk through a p-vector, not a
          // random row of S.
          if (jnn < p) {
            if (myrow == 0)
              sjn_n = A.sd1[jn];
            else if (jn != 0 && jnn != 0)
              sjn_n = A.sd2[jn];
            else
              sjn_n = __ldg(A.S + (size_t)jn * ld + jnn);
          }
        }
        // -- slot-reuse guard, read two steps ahead: the value used now was
        //    loaded two iterations ago (progress only grows, so an early read
        //    that passes is conclusive; a failing one is re-polled below).
        //    Grid: the reader of our publication kDepth steps before the one
        //    at iteration c + 2 must have published since.  Cluster: the
        //    partner of iteration c + 2's publication must have consumed the
        //    step kDepth before it.
        const unsigned long long* rw = rw_next;  // grid: word for this iteration
        const unsigned* rprog = rp_next;         // cluster
        const unsigned rtag = rtag_next;
        rw_next = rw_new;
        rp_next = rp_new;
        rtag_next = rtag_new;
        rw_new = nullptr;
        rp_new = nullptr;
        rtag_new = 0xffffffffu;
        int j3 = p;  // partner of step c + 3
        if (has_row && c + 3 < P) {
          j3 = (myrow == 0) ? (P - (c + 3)) : ring_partner(ring_norm(rr - 4, P), myrow);
          if (c + 3 >= kDepth) {
            if constexpr (CLUSTER) {
              if (j3 < p) {
                rp_new = (const unsigned*)map_rank(prog + (j3 >> cs_log2), j3 & (CS - 1));
                rtag_new = ld_cluster_u32(rp_new);
              }
            } else {
              const int jo = (myrow == 0) ? (P - (c + 3 - kDepth))
                                          : ring_partner(ring_norm(rr - 4 + 2 * kDepth, P), myrow);
              if (jo < p) {
                rw_new = A.mbox + ((size_t)((step + 4u) & (kDepth - 1)) * pe + jo) * MB::kWords;
                rtag_new = MB::read_tag(rw_new);
              }
            }
          }
        }
        // -- wait for the partner
        bool gave_up = false;
        if (!__all_sync(FULL, done)) {
          uint64_t t0 = globaltimer_ns();
          unsigned it = 0;
          while (!__all_sync(FULL, done)) {
            // back off between polls: spinning warps would otherwise crowd the
            // load/store pipe that the working warps need
            if (A.poll_ns) __nanosleep(A.poll_ns);
            if (!done) {
              if constexpr (CLUSTER)
                done = box_read<T>(src, step, wji);
              else
                done = MB::try_read(src, step, wji);
              if (!done && (++it & 63u) == 0) {
                if (ld_relaxed_s32(wc.abort) != 0) {
                  done = gave_up = true;
                } else if (globaltimer_ns() - t0 > wc.timeout_ns) {
                  record_timeout(wc, myrow, (int)(t * P + c));
                  done = gave_up = true;
                }
              }
            }
          }
        }
        if constexpr (CLUSTER) {
          // this row has consumed step `step` (a bye counts as consumed)
          if (has_row) st_cluster_u32(prog + li, step);
        }
        // -- Eq. 3 in S units with W:  x = (s_ii + s_jj) w_ij - W_lo,hi - W_hi,lo
        T delta = (T)0;
        if (paired && !gave_up) {
          const bool i_lo = myrow < j;
          const T wa = i_lo ? pub : wji;  // W_lo,hi
          const T wb = i_lo ? wji : pub;  // W_hi,lo
          const T ss = i_lo ? (s_mine + so) : (so + s_mine);
          const T x = (ss * om - wa) - wb;
          const T sx = soft_threshold(x, lam);
          // most pairs threshold to zero: divide only when needed
          T nw = (T)0;
          if (sx != (T)0) nw = sx / ss;
          delta = nw - om;
          if (delta != (T)0) {
            Orow[j] = nw;
            dmax = fmax(dmax, (double)fabs(delta));
            nact += 1.0;
          }
        }
        // -- next published value: W_i,jn plus every pending update
        if (has_row && more) {
          T v = wA;
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < nA) v = fma_t(pd[k * pst], g[k], v);
          if (dprev != (T)0) v = fma_t(dprev, sprev, v);
          if (delta != (T)0) v = fma_t(delta, sjn, v);
          pub = v;
          const unsigned need = step + 2u - (unsigned)kDepth;  // consumed-through step
          if constexpr (CLUSTER) {
            if (rprog && rtag < need - 1u) {
              uint64_t t0 = globaltimer_ns();
              unsigned it = 0;
              while (ld_cluster_u32(rprog) < need - 1u) {
                if (A.poll_ns) __nanosleep(A.poll_ns);
                if ((++it & 63u) == 0) {
                  if (ld_relaxed_s32(wc.abort) != 0) break;
                  if (globaltimer_ns() - t0 > wc.timeout_ns) {
                    record_timeout(wc, myrow, (int)(t * P + c + 1));
                    break;
                  }
                }
              }
            }
            if (jn < p && !(myrow == A.fault_vertex && t * P + c + 1 == A.fault_step))
              box_store<T>((unsigned long long*)map_rank(
                               box + ((size_t)((step + 1u) & (kDepth - 1)) * cap + (jn >> cs_log2)) * BW,
                               jn & (CS - 1)),
                           step + 1u, pub);
          } else {
            if (rw && rtag < need) {
              uint64_t t0 = globaltimer_ns();
              unsigned it = 0;
              while (MB::read_tag(rw) < need) {
                if (A.poll_ns) __nanosleep(A.poll_ns);
                if ((++it & 63u) == 0) {
                  if (ld_relaxed_s32(wc.abort) != 0) break;
                  if (globaltimer_ns() - t0 > wc.timeout_ns) {
                    record_timeout(wc, myrow, (int)(t * P + c + 1));
                    break;
                  }
                }
              }
            }
            if (!(myrow == A.fault_vertex && t * P + c + 1 == A.fault_step))
              MB::publish(A.mbox + ((size_t)((step + 1u) & (kDepth - 1)) * pe + myrow) * MB::kWords,
                          step + 1u, pub);
          }
        }
        // -- operands of the value published two steps ahead: W_i,jnn and the
        //    S entries of the pending updates in column jnn (loaded now,
        //    consumed in the next step, before any of them can change)
        nA = 0;
        wA = (T)0;
        sprev = (T)0;
        if (has_row && jnn < p) {
          wA = Wrow[jnn];
          nA = cnt;
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < cnt) g[k] = __ldg(A.S + (size_t)pu[k * pst] * ld + jnn);
          if (delta != (T)0) sprev = __ldg(A.S + (size_t)j * ld + jnn);
        }
        dprev = delta;
        if (delta != (T)0) {
          pu[cnt * pst] = j;
          pd[cnt * pst] = delta;
          ++cnt;
        }
        // -- rows whose pending list is full are brought up to date now; the
        //    loads above read W before the flush, matching nA / g[]
        unsigned full = __ballot_sync(FULL, cnt == KC);
        if (full) {
          __syncwarp();
          while (full) {
            const int k = __ffs(full) - 1;
            full &= full - 1;
            const int i = __shfl_sync(FULL, myrow, k);
            flush_row(A.W + (size_t)i * ld, A.S, pu_all + (size_t)wid * KC * R + k,
                      pd_all + (size_t)wid * KC * R + k, pst, KC, ld, lane);
          }
          __syncwarp();
          if (cnt == KC) cnt = 0;
        }
        om = om_n;
        so = so_n;
        sjn = sjn_n;
        j = jn;
        jn = jnn;
        rr -= 2;
        while (rr < 0) rr += P;
      }
      // -- apply every remaining pending update before the diagonal step
      __syncwarp();
      {
        unsigned left = __ballot_sync(FULL, cnt > 0);
        while (left) {
          const int k = __ffs(left) - 1;
          left &= left - 1;
          const int i = __shfl_sync(FULL, myrow, k);
          const int n = __shfl_sync(FULL, cnt, k);
          flush_row(A.W + (size_t)i * ld, A.S, pu_all + (size_t)wid * KC * R + k,
                    pd_all + (size_t)wid * KC * R + k, pst, n, ld, lane);
        }
        __syncwarp();
      }
      // -- diagonal step (Eq. 2 divided by n): c_i = W_ii - w_ii s_ii,
      //    w_ii <- (-c_i + sqrt(c_i^2 + 4 s_ii)) / (2 s_ii), W_i += dw S_i
      T dd = (T)0;
      if (has_row && ld_relaxed_s32(wc.abort) == 0) {
        const double sii = A.sdiag64[myrow];
        const double wii = (double)Wrow[myrow];
        const double oii = MIXED ? A.omdiag64[myrow] : (double)Orow[myrow];
        const double ci = wii - oii * sii;
        const double nw = (-ci + sqrt(ci * ci + 4.0 * sii)) / (2.0 * sii);
        if (MIXED) A.omdiag64[myrow] = nw;
        Orow[myrow] = (T)nw;
        dd = (T)(nw - oii);
        dmax = fmax(dmax, fabs(nw - oii));
      }
      unsigned act = __ballot_sync(FULL, dd != (T)0);
      while (act) {
        const int k = __ffs(act) - 1;
        act &= act - 1;
        const int i = __shfl_sync(FULL, myrow, k);
        const T d = __shfl_sync(FULL, dd, k);
        axpy_row(A.W + (size_t)i * ld, A.S + (size_t)i * ld, d, ld, lane);
      }
      __syncwarp();
    }

    // ---------------- fused objective / KKT pass over the upper triangle
    if constexpr (CLUSTER)
      cluster_sync_all();
    else
      group_barrier(A.barrier, gen, G, wc, 1000000 + t, cta);
    double v[kParts];
#pragma unroll
    for (int k = 0; k < kParts; ++k) v[k] = 0.0;
    v[kPartDelta] = dmax;
    v[kPartActive] = nact;
    {
      // Work unit: an 8-row chunk of a 32 x 32 tile (ta <= tb) of the upper
      // triangle.  Lane l takes column j = tb*32 + l: W_ij comes from row i
      // (coalesced across lanes), W_ji from row j as one 8-element vector, so
      // G_ij = W_ij + W_ji pairs up without a transpose.
      using VT = Vec16<T>;
      using V = typename VT::V;
      constexpr int NV = 8 / VT::N;
      const int nb = (p + kTile - 1) / kTile;
      const double lamd = lam_cur;
      const float lamf = (float)lam_cur;
      const int units = nb * nb * 4;
      const int gwarps = G * (blockDim.x >> 5);
      for (int u = cta * (blockDim.x >> 5) + wid; u < units; u += gwarps) {
        const int tau = u >> 2, r0 = (u & 3) * 8;
        const int ta = tau / nb, tb = tau % nb;
        if (ta > tb) continue;
        const int j = tb * kTile + lane;
        const int i0 = ta * kTile + r0;
        if (i0 >= p) continue;
        T w1[8], om8[8], wt[8];
        const bool jv = j < p;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = i0 + r;
          const bool ok = jv && i < p;
          w1[r] = ok ? __ldcg(A.W + (size_t)i * ld + j) : (T)0;
          om8[r] = ok ? __ldcg(A.Om + (size_t)i * ld + j) : (T)0;
        }
        if (jv) {
          const V* src = reinterpret_cast<const V*>(A.W + (size_t)j * ld + i0);
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            V x = __ldcg(src + q);
            if constexpr (VT::N == 4) {
              wt[4 * q + 0] = ((const float*)&x)[0];
              wt[4 * q + 1] = ((const float*)&x)[1];
              wt[4 * q + 2] = ((const float*)&x)[2];
              wt[4 * q + 3] = ((const float*)&x)[3];
            } else {
              wt[2 * q + 0] = ((const double*)&x)[0];
              wt[2 * q + 1] = ((const double*)&x)[1];
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < 8; ++r) wt[r] = (T)0;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = i0 + r;
          if (!jv || i >= p) continue;
          if (i < j) {
            const T om_t = om8[r];
            // FP32 screen: a zero entry whose |G_ij| is clearly below lambda
            // has residual exactly 0 (the margin covers the FP32 rounding of
            // G); every other entry is evaluated in FP64.
            const float w1f = (float)w1[r], w2f = (float)wt[r];
            const float gf = w1f + w2f;
            if (om_t == (T)0 && fabsf(gf) <= lamf - 1e-5f * (1.0f + fabsf(w1f) + fabsf(w2f)))
              continue;
            const double om = (double)om_t;
            const double g = (double)w1[r] + (double)wt[r];
            double res;
            if (om > 0.0)
              res = fabs(g + lamd);
            else if (om < 0.0)
              res = fabs(g - lamd);
            else
              res = fmax(fabs(g) - lamd, 0.0);
            v[kPartKkt] = fmax(v[kPartKkt], res);
            v[kPartQuad] += om * g;
            v[kPartPen] += fabs(om);
            if (!isfinite(g) || !isfinite(om)) v[kPartBad] += 1.0;
          } else if (i == j) {
            const double wii = (double)w1[r];
            const double oii = MIXED ? __ldcg(A.omdiag64 + i) : (double)om8[r];
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
    block_reduce_parts(v, A.partials, red, cta);
    if constexpr (CLUSTER)
      cluster_sync_all();
    else
      group_barrier(A.barrier, gen, G, wc, 2000000 + t, cta);

    // ---------------- every CTA reduces the partials identically
    if (threadIdx.x == 0) {
      double kkt = 0.0, quad = 0.0, pen = 0.0, lg = 0.0, dl = 0.0, ac = 0.0, bad = 0.0;
      for (int b = 0; b < (int)G; ++b) {
        const double* q = A.partials + (size_t)b * kParts;
        kkt = fmax(kkt, __ldcg(q + kPartKkt));
        quad += __ldcg(q + kPartQuad);
        pen += __ldcg(q + kPartPen);
        lg += __ldcg(q + kPartLog);
        dl = fmax(dl, __ldcg(q + kPartDelta));
        ac += __ldcg(q + kPartActive);
        bad += __ldcg(q + kPartBad);
      }
      const double obj = -lg + 0.5 * quad + lam_cur * pen;
      const bool aborted = ld_relaxed_s32(wc.abort) != 0;
      const bool nonfinite = bad > 0.0 || !isfinite(obj) || !isfinite(kkt);
      const int t_count = BATCH ? t_lam : t;
      const int sweeps_done = do_sweep ? t_count + 1 : t_count;
      if (do_sweep && first_delta == 0 && dl < A.delta_tol) first_delta = sweeps_done;
      bool conv = (A.stop_rule == 1) ? (do_sweep && dl < A.tol) : (kkt <= A.tol);
      // stall: the KKT residual has not dropped by 10% for 4 sweeps (FP32
      // phase at its rounding floor); the host then switches to FP64
      bool stalled = false;
      if (do_sweep) {
        if (kkt < 0.9 * best_kkt) {
          best_kkt = kkt;
          since_best = 0;
        } else if (++since_best >= 4 && A.stall_stop) {
          stalled = true;
        }
      }
      s_res[kResSweeps] = sweeps_done;
      s_res[kResKkt] = kkt;
      s_res[kResObj] = obj;
      s_res[kResDelta] = dl;
      s_res[kResActive] = ac * 0.5;  // each pair is counted by both owners
      s_res[kResFirstDelta] = first_delta;
      s_res[kResStatus] = aborted ? 3.0 : (nonfinite ? 2.0 : (conv ? 0.0 : (stalled ? 4.0 : 1.0)));
      s_stop = (aborted || nonfinite || conv || stalled || A.kkt_only || sweeps_done >= A.n_sweeps)
                   ? 1
                   : 0;
      if constexpr (BATCH) {
        // the lambda is finished; the problem stops after the last one (or
        // on an abort / a non-finite value) and otherwise moves to the next
        // (a lambda that ends on the stall rule ends the walk when asked: the
        // host polishes it in FP64 and resumes after it; its support is the
        // polished one, so it is not counted here)
        s_lam_end = s_stop;
        const bool brk = stalled && A.stall_break;
        s_lam_count = s_stop && !brk;
        if (s_stop && !aborted && !nonfinite && !brk && kl + 1 < A.n_lambda) s_stop = 0;
        if (cta == 0 && s_lam_end)
          for (int k = 0; k < kRes; ++k) A.result[(size_t)kl * kRes + k] = s_res[k];
      }
      if (cta == 0) {
        if (do_sweep && t < A.hist_len) {
          double* h = A.hist + (size_t)t * kHist;
          h[0] = dl;
          h[1] = kkt;
          h[2] = obj;
          h[3] = ac * 0.5;
        }
        if (!BATCH && s_stop)
          for (int k = 0; k < kRes; ++k) A.result[k] = s_res[k];
      }
    }
    __syncthreads();
    if constexpr (BATCH) {
      if (s_lam_end) {
        // support of this lambda's solution over the rows this warp owns (no
        // other warp writes them, so no barrier is needed before the next
        // lambda's sweeps)
        // (warp-uniform conditions only: the loop below shuffles)
        const bool live = __shfl_sync(FULL, ld_relaxed_s32(wc.abort) == 0 ? 1 : 0, 0) != 0;
        if (A.batch_cnt && s_lam_count && row_warp && live) {
          float* cnt_k = A.batch_cnt + (size_t)kl * p * p;
          unsigned own = __ballot_sync(FULL, has_row);
          while (own) {
            const int k = __ffs(own) - 1;
            own &= own - 1;
            const int i = __shfl_sync(FULL, myrow, k);
            const T* orow = A.Om + (size_t)i * ld;
            for (int x = lane; x < p; x += 32)
              if (orow[x] != (T)0) atomicAdd(cnt_k + (size_t)i * p + x, 1.0f);
          }
        }
        if (!s_stop) {
          ++kl;
          lam_cur = A.lambdas[kl];
          lam = (T)lam_cur;
          best_kkt = 1e300;
          since_best = 0;
          first_delta = 0;
          t_lam = -1;
        }
      }
      ++t_lam;
    }
    if (s_stop) break;
    ++t;
  }
}

template <typename T, bool MIXED, bool CLUSTER>
cudaError_t launch_sweep_impl(const SweepArgs<T>& args, int grid, int block, cudaStream_t st) {
  const size_t dyn = sweep_dyn_smem(sizeof(T), args.row_warps, args.rows_per_warp, CLUSTER);
  const void* fn = (const void*)k_sweep<T, MIXED, CLUSTER, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  note_launches(1);
  if constexpr (CLUSTER) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = grid;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep<T, MIXED, CLUSTER, false>, args);
  } else {
    void* kargs[] = {(void*)&args};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), kargs, dyn, st);
  }
}

template <typename T, bool MIXED>
cudaError_t sweep_occupancy_impl(int block, int* blocks_per_sm) {
  const size_t dyn = sweep_dyn_smem(sizeof(T), block / 32, 32, false);
  cudaError_t e = cudaFuncSetAttribute((const void*)k_sweep<T, MIXED, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                       k_sweep<T, MIXED, false, false>, block, dyn);
}

// Largest cluster the cluster variant can launch with (a power of two <= 16),
// for one CTA of `block` threads holding `rows` rows.
template <typename T, bool MIXED>
cudaError_t sweep_cluster_size_impl(int block, int row_warps, int rows_per_warp, int* cs) {
  const size_t dyn = sweep_dyn_smem(sizeof(T), row_warps, rows_per_warp, true);
  const void* fn = (const void*)k_sweep<T, MIXED, true, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  *cs = 0;
  for (int c = 16; c >= 2; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k_sweep<T, MIXED, true, false>, &cfg);
    if (e == cudaSuccess && n >= 1) {
      *cs = c;
      return cudaSuccess;
    }
    cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_sweep(const SweepArgs<double>& a, int grid, int block, bool cluster,
                         cudaStream_t st) {
  return cluster ? launch_sweep_impl<double, false, true>(a, grid, block, st)
                 : launch_sweep_impl<double, false, false>(a, grid, block, st);
}
cudaError_t launch_sweep(const SweepArgs<float>& a, int grid, int block, bool cluster,
                         cudaStream_t st) {
  return cluster ? launch_sweep_impl<float, true, true>(a, grid, block, st)
                 : launch_sweep_impl<float, true, false>(a, grid, block, st);
}
template <typename T, bool MIXED>
cudaError_t launch_sweep_batch_impl(const SweepArgs<T>& args, int grid, int block, cudaStream_t st) {
  const size_t dyn = sweep_dyn_smem(sizeof(T), args.row_warps, args.rows_per_warp, false);
  const void* fn = (const void*)k_sweep<T, MIXED, false, true>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  note_launches(1);
  void* kargs[] = {(void*)&args};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), kargs, dyn, st);
}

cudaError_t launch_sweep_batch(const SweepArgs<double>& a, int grid, int block, cudaStream_t st) {
  return launch_sweep_batch_impl<double, false>(a, grid, block, st);
}
cudaError_t launch_sweep_batch(const SweepArgs<float>& a, int grid, int block, cudaStream_t st) {
  return launch_sweep_batch_impl<float, true>(a, grid, block, st);
}

cudaError_t sweep_occupancy(bool mixed, int block, int* blocks_per_sm) {
  return mixed ? sweep_occupancy_impl<float, true>(block, blocks_per_sm)
               : sweep_occupancy_impl<double, false>(block, blocks_per_sm);
}
cudaError_t sweep_cluster_size(bool mixed, int block, int row_warps, int rows_per_warp, int* cs) {
  return mixed ? sweep_cluster_size_impl<float, true>(block, row_warps, rows_per_warp, cs)
               : sweep_cluster_size_impl<double, false>(block, row_warps, rows_per_warp, cs);
}

// ---------------------------------------------------------------------------
// W = Omega S in FP64 for a sparse Omega (one warp per row): the nonzeros of
// row i are gathered into shared memory, then W_i = sum_u w_iu S_u with FP64
// accumulation.  Used to rebuild W at warm starts and before FP64 polishing.
// ---------------------------------------------------------------------------
constexpr int kRefreshWarps = 8;
constexpr int kRefreshCap = 256;

__global__ void __launch_bounds__(kRefreshWarps * 32) k_refresh_w(const double* __restrict__ Om,
                                                                  const double* __restrict__ S,
                                                                  double* __restrict__ W, int p,
                                                                  int ld) {
  __shared__ int nz_i[kRefreshWarps][kRefreshCap];
  __shared__ double nz_v[kRefreshWarps][kRefreshCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int row = blockIdx.x * kRefreshWarps + wid; row < p; row += gridDim.x * kRefreshWarps) {
    const double* orow = Om + (size_t)row * ld;
    double* wrow = W + (size_t)row * ld;
    int scan = 0;
    bool first = true;
    while (scan < ld || first) {
      // gather up to kRefreshCap nonzeros starting at `scan`
      int cnt = 0;
      while (scan < ld && cnt < kRefreshCap) {
        const int u = scan + lane;
        const double v = (u < ld) ? orow[u] : 0.0;
        const bool nz = v != 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        const int room = kRefreshCap - cnt;
        const int take = min(__popc(m), room);
        // lanes beyond `room` are left for the next batch
        const int rank = __popc(m & ((1u << lane) - 1u));
        if (nz && rank < take) {
          nz_i[wid][cnt + rank] = u;
          nz_v[wid][cnt + rank] = v;
        }
        if (take < __popc(m)) {
          // resume at the first nonzero that did not fit
          unsigned rest = m;
          for (int q = 0; q < take; ++q) rest &= rest - 1;
          scan += __ffs(rest) - 1;
          cnt += take;
          break;
        }
        cnt += take;
        scan += 32;
      }
      __syncwarp();
      for (int c0 = 0; c0 < ld; c0 += 128) {
        double acc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int col = c0 + lane + 32 * m;
          acc[m] = (!first && col < ld) ? wrow[col] : 0.0;
        }
        for (int q = 0; q < cnt; ++q) {
          const double w = nz_v[wid][q];
          const double* srow = S + (size_t)nz_i[wid][q] * ld;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int col = c0 + lane + 32 * m;
            if (col < ld) acc[m] = fma(w, srow[col], acc[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int col = c0 + lane + 32 * m;
          if (col < ld) wrow[col] = acc[m];
        }
      }
      __syncwarp();
      first = false;
    }
  }
}

cudaError_t launch_refresh_w(const double* Om, const double* S, double* W, int p, int ld, int sms,
                             cudaStream_t st) {
  int grid = (p + kRefreshWarps - 1) / kRefreshWarps;
  if (grid > sms * 8) grid = sms * 8;
  k_refresh_w<<<grid, kRefreshWarps * 32, 0, st>>>(Om, S, W, p, ld);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace concord
