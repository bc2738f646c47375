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
                                                   double (*red)[kParts]) {
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
      out[(size_t)blockIdx.x * kParts + k] = x;
    }
  }
  __syncthreads();
}

template <typename T, bool MIXED>
__global__ void __launch_bounds__(kSweepThreads, 1) k_sweep(const SweepArgs<T> a) {
  using MB = Mailbox<T>;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int TW = gridDim.x * wpb;
  const int p = a.p, P = a.P, ld = a.ld, D = a.depth;
  const int pe = P + 1;
  const int myrow = gw + lane * TW;
  const bool has_row = lane < a.rows_per_warp && myrow < p;
  const T lam = (T)a.lambda;
  const WaitCtl& wc = a.wait;

  __shared__ T t1[kTile][kTile + 1];
  __shared__ T t2[kTile][kTile + 1];
  __shared__ double red[kSweepThreads / 32][kParts];
  __shared__ int s_stop;
  __shared__ double s_res[kRes];

  unsigned gen = 0;
  int first_delta = 0;
  int t = 0;
  T* __restrict__ Wrow = a.W + (size_t)(has_row ? myrow : 0) * ld;
  T* __restrict__ Orow = a.Om + (size_t)(has_row ? myrow : 0) * ld;
  const T s_mine = has_row ? a.sdiag[myrow] : (T)1;

  for (;;) {
    const bool do_sweep = !a.kkt_only && t < a.n_sweeps;
    double dmax = 0.0, nact = 0.0;
    if (do_sweep) {
      // value to publish at colour 0: W_i,partner(i,0)
      int j = has_row ? cm_partner(myrow, 0, P) : p;
      T pub = (has_row && j < p) ? Wrow[j] : (T)0;
      for (int c = 0; c < P; ++c) {
        const unsigned step = a.tag_base + (unsigned)(t * P + c);
        const int slot = (int)(step % (unsigned)D);
        const bool paired = has_row && j < p;
        // -- slot reuse: our publication D steps ago must have been consumed,
        //    i.e. its reader has published at least step-D+1.
        if (has_row && step >= a.tag_base + (unsigned)D) {
          const unsigned old = step - (unsigned)D;
          const int jo = cm_partner(myrow, (int)((old - a.tag_base) % (unsigned)P), P);
          if (jo < p) {
            const unsigned long long* ack =
                a.mbox + ((size_t)((old + 1u) % (unsigned)D) * pe + jo) * MB::kWords;
            if (MB::read_tag(ack) < old + 1u) {
              uint64_t t0 = globaltimer_ns();
              unsigned it = 0;
              while (MB::read_tag(ack) < old + 1u) {
                if ((++it & 63u) == 0) {
                  if (ld_volatile_s32(wc.abort) != 0) break;
                  if (globaltimer_ns() - t0 > wc.timeout_ns) {
                    record_timeout(wc, myrow, (int)(t * P + c));
                    break;
                  }
                }
              }
            }
          }
        }
        // -- publish W_ij for this step (a bye publishes a placeholder so the
        //    slot-reuse check above always has a later tag to look for)
        if (has_row && !(myrow == a.fault_vertex && t * P + c == a.fault_step))
          MB::publish(a.mbox + ((size_t)slot * pe + myrow) * MB::kWords, step, pub);
        // -- operands of this step and of the next step's published value
        T om = (T)0, s_other = (T)1;
        int jn = p;
        T wn = (T)0, sjn = (T)0;
        if (paired) {
          om = Orow[j];
          s_other = a.sdiag[j];
        }
        if (has_row && c + 1 < P) {
          jn = cm_partner(myrow, c + 1, P);
          if (jn < p) {
            wn = Wrow[jn];
            if (paired) sjn = __ldg(a.S + (size_t)j * ld + jn);
          }
        }
        // -- wait for the partner's W_ji
        T wji = (T)0;
        bool gave_up = false;  // this lane's wait ended by abort / timeout
        bool done = !paired;
        if (paired) done = MB::try_read(a.mbox + ((size_t)slot * pe + j) * MB::kWords, step, wji);
        if (!__all_sync(FULL, done)) {
          uint64_t t0 = globaltimer_ns();
          unsigned it = 0;
          while (!__all_sync(FULL, done)) {
            if (!done) {
              done = MB::try_read(a.mbox + ((size_t)slot * pe + j) * MB::kWords, step, wji);
              if (!done && (++it & 63u) == 0) {
                if (ld_volatile_s32(wc.abort) != 0) {
                  done = gave_up = true;
                } else if (globaltimer_ns() - t0 > wc.timeout_ns) {
                  record_timeout(wc, myrow, (int)(t * P + c));
                  done = gave_up = true;
                }
              }
            }
          }
        }
        // -- Eq. 3 in S units with W:  x = (s_ii + s_jj) w_ij - W_lo,hi - W_hi,lo
        T delta = (T)0;
        if (paired) {
          const bool i_lo = myrow < j;
          const T wa = i_lo ? pub : wji;  // W_lo,hi
          const T wb = i_lo ? wji : pub;  // W_hi,lo
          const T ss = i_lo ? (s_mine + s_other) : (s_other + s_mine);
          const T x = (ss * om - wa) - wb;
          const T nw = soft_threshold(x, lam) / ss;
          delta = gave_up ? (T)0 : nw - om;
          if (delta != (T)0) {
            Orow[j] = nw;
            dmax = fmax(dmax, (double)fabs(delta));
            nact += 1.0;
          }
        }
        // next published value, formed with the same FMA as the row update
        pub = (delta != (T)0) ? fma_t(delta, sjn, wn) : wn;
        // -- row updates of the active pairs owned by this warp
        unsigned act = __ballot_sync(FULL, delta != (T)0);
        while (act) {
          const int k = __ffs(act) - 1;
          act &= act - 1;
          const int i = __shfl_sync(FULL, myrow, k);
          const int jj = __shfl_sync(FULL, j, k);
          const T d = __shfl_sync(FULL, delta, k);
          axpy_row(a.W + (size_t)i * ld, a.S + (size_t)jj * ld, d, ld, lane);
        }
        __syncwarp();
        j = jn;
      }
      // -- diagonal step (Eq. 2 divided by n): c_i = W_ii - w_ii s_ii,
      //    w_ii <- (-c_i + sqrt(c_i^2 + 4 s_ii)) / (2 s_ii), W_i += dw S_i
      T dd = (T)0;
      if (has_row && ld_volatile_s32(wc.abort) == 0) {
        const double sii = a.sdiag64[myrow];
        const double wii = (double)Wrow[myrow];
        const double oii = MIXED ? a.omdiag64[myrow] : (double)Orow[myrow];
        const double ci = wii - oii * sii;
        const double nw = (-ci + sqrt(ci * ci + 4.0 * sii)) / (2.0 * sii);
        if (MIXED) {
          a.omdiag64[myrow] = nw;
          Orow[myrow] = (T)nw;
        } else {
          Orow[myrow] = (T)nw;
        }
        dd = (T)(nw - oii);
        dmax = fmax(dmax, fabs(nw - oii));
      }
      unsigned act = __ballot_sync(FULL, dd != (T)0);
      while (act) {
        const int k = __ffs(act) - 1;
        act &= act - 1;
        const int i = __shfl_sync(FULL, myrow, k);
        const T d = __shfl_sync(FULL, dd, k);
        axpy_row(a.W + (size_t)i * ld, a.S + (size_t)i * ld, d, ld, lane);
      }
      __syncwarp();
    }

    // ---------------- fused objective / KKT pass over the upper triangle
    grid_barrier(a.barrier, gen, wc, 1000000 + t);
    double v[kParts];
#pragma unroll
    for (int k = 0; k < kParts; ++k) v[k] = 0.0;
    v[kPartDelta] = dmax;
    v[kPartActive] = nact;
    const int nb = (p + kTile - 1) / kTile;
    const double lamd = a.lambda;
    for (int tau = blockIdx.x; tau < nb * nb; tau += gridDim.x) {
      const int ta = tau / nb, tb = tau % nb;
      if (ta > tb) continue;
      for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = e >> 5, cc = e & 31;
        const int i1 = ta * kTile + r, j1 = tb * kTile + cc;
        const int i2 = tb * kTile + r, j2 = ta * kTile + cc;
        // L2-only loads: rows written by other SMs must not come from a stale L1 line
        t1[r][cc] = (i1 < p && j1 < p) ? __ldcg(a.W + (size_t)i1 * ld + j1) : (T)0;
        t2[r][cc] = (i2 < p && j2 < p) ? __ldcg(a.W + (size_t)i2 * ld + j2) : (T)0;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = e >> 5, cc = e & 31;
        const int i = ta * kTile + r, j = tb * kTile + cc;
        if (i >= p || j >= p) continue;
        if (ta < tb || r < cc) {
          const double om = (double)__ldcg(a.Om + (size_t)i * ld + j);
          const double g = (double)t1[r][cc] + (double)t2[cc][r];
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
        } else if (r == cc) {
          const double wii = (double)t1[r][r];
          const double oii = MIXED ? __ldcg(a.omdiag64 + i) : (double)__ldcg(a.Om + (size_t)i * ld + i);
          if (oii > 0.0 && isfinite(wii) && isfinite(oii)) {
            v[kPartKkt] = fmax(v[kPartKkt], fabs(wii - 1.0 / oii));
            v[kPartQuad] += oii * wii;
            v[kPartLog] += log(oii);
          } else {
            v[kPartBad] += 1.0;
          }
        }
      }
      __syncthreads();
    }
    block_reduce_parts(v, a.partials, red);
    grid_barrier(a.barrier, gen, wc, 2000000 + t);

    // ---------------- every CTA reduces the partials identically
    if (threadIdx.x == 0) {
      double kkt = 0.0, quad = 0.0, pen = 0.0, lg = 0.0, dl = 0.0, ac = 0.0, bad = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        const double* q = a.partials + (size_t)b * kParts;
        kkt = fmax(kkt, __ldcg(q + kPartKkt));
        quad += __ldcg(q + kPartQuad);
        pen += __ldcg(q + kPartPen);
        lg += __ldcg(q + kPartLog);
        dl = fmax(dl, __ldcg(q + kPartDelta));
        ac += __ldcg(q + kPartActive);
        bad += __ldcg(q + kPartBad);
      }
      const double obj = -lg + 0.5 * quad + lamd * pen;
      const bool aborted = ld_volatile_s32(wc.abort) != 0;
      const bool nonfinite = bad > 0.0 || !isfinite(obj) || !isfinite(kkt);
      const int sweeps_done = do_sweep ? t + 1 : t;
      if (do_sweep && first_delta == 0 && dl < a.delta_tol) first_delta = sweeps_done;
      bool conv = (a.stop_rule == 1) ? (do_sweep && dl < a.tol) : (kkt <= a.tol);
      s_res[kResSweeps] = sweeps_done;
      s_res[kResKkt] = kkt;
      s_res[kResObj] = obj;
      s_res[kResDelta] = dl;
      s_res[kResActive] = ac * 0.5;  // each pair is counted by both owners
      s_res[kResFirstDelta] = first_delta;
      s_res[kResStatus] = aborted ? 3.0 : (nonfinite ? 2.0 : (conv ? 0.0 : 1.0));
      s_stop = (aborted || nonfinite || conv || a.kkt_only || sweeps_done >= a.n_sweeps) ? 1 : 0;
      if (blockIdx.x == 0) {
        if (do_sweep && t < a.hist_len) {
          double* h = a.hist + (size_t)t * kHist;
          h[0] = dl;
          h[1] = kkt;
          h[2] = obj;
          h[3] = ac * 0.5;
        }
        if (s_stop)
          for (int k = 0; k < kRes; ++k) a.result[k] = s_res[k];
      }
    }
    __syncthreads();
    if (s_stop) break;
    ++t;
  }
}

template <typename T, bool MIXED>
cudaError_t launch_sweep_impl(const SweepArgs<T>& args, int grid, int block, cudaStream_t st) {
  void* kargs[] = {(void*)&args};
  note_launches(1);
  return cudaLaunchCooperativeKernel((const void*)k_sweep<T, MIXED>, dim3(grid), dim3(block), kargs,
                                     0, st);
}

template <typename T, bool MIXED>
cudaError_t sweep_occupancy_impl(int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sweep<T, MIXED>, block, 0);
}

cudaError_t launch_sweep(const SweepArgs<double>& a, int grid, int block, cudaStream_t st) {
  return launch_sweep_impl<double, false>(a, grid, block, st);
}
cudaError_t launch_sweep(const SweepArgs<float>& a, int grid, int block, cudaStream_t st) {
  return launch_sweep_impl<float, true>(a, grid, block, st);
}
cudaError_t sweep_occupancy(bool mixed, int block, int* blocks_per_sm) {
  return mixed ? sweep_occupancy_impl<float, true>(block, blocks_per_sm)
               : sweep_occupancy_impl<double, false>(block, blocks_per_sm);
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
