// Device helpers shared by the CONCORD-PCD kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace concord {

constexpr int kTile = 32;  // row-stride granularity (elements) and KKT tile edge

// ---------------------------------------------------------------------------
// Circle-method partner, closed form (Section 3.2, Algorithm 1).
//
// Algorithm 1 keeps vertex 1 fixed and, after every colour, rotates positions
// 2..pe by one place; colour k pairs position q with position pe-q+1.  In
// 0-based labels with P = pe - 1 colours: vertex v >= 1 sits at ring index
// (v - 1 + c) mod P during colour c; ring index P-1 is the position facing
// vertex 0; ring indices r and P-2-r face each other.  Solving for the vertex
// at the facing index gives w = ((-v - 1 - 2c) mod P) + 1, which equals v
// exactly when v faces vertex 0.  For odd p the extra vertex p (1-based p+1)
// is a real ring member here; whoever faces it sits the colour out.
// ---------------------------------------------------------------------------
__host__ __device__ inline int cm_partner(int v, int c, int P) {
  if (v == 0) return (P - 1 - c) % P + 1;
  int w = (-v - 1 - 2 * c) % P;
  if (w < 0) w += P;
  w += 1;
  return (w == v) ? 0 : w;
}

// ---------------------------------------------------------------------------
// Bounded waits.  Every spin in this library ends: on success, when the
// shared abort word becomes non-zero, or when %globaltimer passes the limit
// (then it records the code and where it gave up, and returns false).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Mailbox words use relaxed GPU-scope accesses: they are served by L2 (the
// GPU's point of coherence), never by a stale L1 line, and need no system-
// scope coherence.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void ld_relaxed_v2u64(const unsigned long long* p,
                                                 unsigned long long& a,
                                                 unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(a), "=l"(b)
               : "l"(p)
               : "memory");
}

__device__ __forceinline__ void st_relaxed_v2u64(unsigned long long* p, unsigned long long a,
                                                 unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b)
               : "memory");
}

// Abort codes written into the shared abort word.
constexpr int kAbortTimeout = 1;

struct WaitCtl {
  int* abort;            // shared abort word (0 = running)
  int* info;             // [0] vertex, [1] step of the first wait that ran out
  uint64_t timeout_ns;   // per-wait limit
};

__device__ __forceinline__ void record_timeout(const WaitCtl& w, int vertex, int step) {
  if (atomicCAS(w.abort, 0, kAbortTimeout) == 0) {
    w.info[0] = vertex;
    w.info[1] = step;
  }
}

// ---------------------------------------------------------------------------
// Per-vertex mailboxes (one scalar per vertex per colour step).
//
// Slot layout: depth D ring indexed by step mod D, then by vertex.  A 32-bit
// value travels with its 32-bit step tag in one 64-bit word; a 64-bit value
// travels as two words (tag|hi, tag|lo), each single-copy atomic, accepted
// only when both tags match.  No other data crosses between the two owners
// of a pair, so no release/acquire ordering is needed beyond the atomic word.
// ---------------------------------------------------------------------------
template <typename T>
struct Mailbox;

template <>
struct Mailbox<float> {
  static constexpr int kWords = 1;
  __device__ static void publish(unsigned long long* slot, unsigned tag, float v) {
    st_relaxed_u64(slot, ((unsigned long long)tag << 32) | __float_as_uint(v));
  }
  __device__ static bool try_read(const unsigned long long* slot, unsigned tag, float& v) {
    unsigned long long w = ld_relaxed_u64(slot);
    v = __uint_as_float((unsigned)(w & 0xffffffffull));
    return (unsigned)(w >> 32) == tag;
  }
  __device__ static unsigned read_tag(const unsigned long long* slot) {
    return (unsigned)(ld_relaxed_u64(slot) >> 32);
  }
};

template <>
struct Mailbox<double> {
  static constexpr int kWords = 2;
  __device__ static void publish(unsigned long long* slot, unsigned tag, double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    unsigned long long t = (unsigned long long)tag << 32;
    st_relaxed_v2u64(slot, t | (b >> 32), t | (b & 0xffffffffull));
  }
  __device__ static bool try_read(const unsigned long long* slot, unsigned tag, double& v) {
    unsigned long long hi, lo;
    ld_relaxed_v2u64(slot, hi, lo);
    unsigned long long b = ((hi & 0xffffffffull) << 32) | (lo & 0xffffffffull);
    v = __longlong_as_double((long long)b);
    return (unsigned)(hi >> 32) == tag && (unsigned)(lo >> 32) == tag;
  }
  __device__ static unsigned read_tag(const unsigned long long* slot) {
    return (unsigned)(ld_relaxed_u64(slot) >> 32);
  }
};

// ---------------------------------------------------------------------------
// Barrier of `count` co-resident CTAs (a cooperative launch, or a group of
// its CTAs with their own counter).  `gen` counts the barriers this group has
// passed; the counter is zeroed before the launch.  Returns with every CTA of
// the group past the barrier or with the abort word set; a wait that runs out
// records -1 - who (the CTA) and `where`.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void group_barrier(unsigned* counter, unsigned& gen, unsigned count,
                                              const WaitCtl& w, int where, int who) {
  __syncthreads();
  ++gen;
  if (threadIdx.x == 0) {
    // the release add publishes the CTA's writes (ordered before it by the
    // CTA barrier); the acquire load that sees the last arrival makes every
    // other CTA's writes visible to the CTA after its closing barrier
    red_release_add_u32(counter, 1u);
    const unsigned target = gen * count;
    uint64_t t0 = globaltimer_ns();
    unsigned it = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++it & 15u) == 0) {
        if (ld_relaxed_s32(w.abort) != 0) break;
        if (globaltimer_ns() - t0 > w.timeout_ns) {
          record_timeout(w, -1 - who, where);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// One round of a group of `count` CTAs that also agree on whether any of
// them set a flag: every CTA adds 1 (+ 2^32 when its flag is set) to the
// round's own 64-bit slot (zeroed before the round) with a release add and
// waits, with acquire loads, until all `count` have arrived -- the arrival
// count and the flags travel together, so the round costs one atomic and
// one wait.  Every CTA reads the same complete sum.  A wait that runs out
// (or an abort) records -1 - who and `where` and reports the flag as set.
__device__ __forceinline__ bool round_barrier_any(unsigned long long* slot, unsigned count,
                                                  bool flag, const WaitCtl& w, int where,
                                                  int who) {
  __shared__ int s_any;
  const bool f = __syncthreads_or(flag) != 0;
  if (threadIdx.x == 0) {
    const unsigned long long add = 1ull + (f ? (1ull << 32) : 0ull);
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(slot), "l"(add) : "memory");
    const uint64_t t0 = globaltimer_ns();
    unsigned it = 0;
    int any = 1;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(slot) : "memory");
      if ((unsigned)(v & 0xffffffffull) >= count) {
        any = (v >> 32) != 0ull ? 1 : 0;
        break;
      }
      if ((++it & 15u) == 0) {
        if (ld_relaxed_s32(w.abort) != 0) break;
        if (globaltimer_ns() - t0 > w.timeout_ns) {
          record_timeout(w, -1 - who, where);
          break;
        }
      }
    }
    s_any = any;
  }
  __syncthreads();
  return s_any != 0;
}

// The whole grid (every CTA of a cooperative launch) as one group.
__device__ __forceinline__ void grid_barrier(unsigned* counter, unsigned& gen,
                                             const WaitCtl& w, int where) {
  group_barrier(counter, gen, gridDim.x, w, where, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// Helpers of the screened sweep and the sparse polish.
// ---------------------------------------------------------------------------
// Colour step (0-based) at which the circle method pairs i < j (Section 3.2,
// Algorithm 1): solving the closed form of cm_partner for the colour gives
// 2c = -(i + j) (mod P) for i >= 1, and c = P - j for i = 0.  P is odd, so
// halving mod P is n / 2 for even n and (n + P) / 2 for odd n.
__device__ __forceinline__ int pair_step(int i, int j, int P) {
  if (i == 0) return P - j;
  int s = i + j;  // i, j <= P, so s < 2P
  if (s >= P) s -= P;
  if (s >= P) s -= P;
  const int neg = s == 0 ? 0 : P - s;
  return (neg & 1) ? (neg + P) >> 1 : neg >> 1;
}

template <typename T>
__device__ __forceinline__ T soft(T x, T tau) {
  T a = fabs(x) - tau;
  if (!(a > (T)0)) return (T)0;
  return x > (T)0 ? a : -a;
}

// KKT residual term of an off-diagonal pair (absolute, S units) with
// G = W_ij + W_ji in FP64.
__device__ __forceinline__ double kkt_offdiag(double om, double g, double lam) {
  if (om > 0.0) return fabs(g + lam);
  if (om < 0.0) return fabs(g - lam);
  return fmax(fabs(g) - lam, 0.0);
}

__device__ __forceinline__ int ldi(const int* p) { return __ldcg(p); }

}  // namespace concord
