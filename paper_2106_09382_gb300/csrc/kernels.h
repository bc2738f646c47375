// Kernel entry points and argument blocks shared by the host API (capi.cu)
// and the kernel translation units.  Internal: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace concord {

// Records `msg` as the calling thread's concord_last_error() text and
// returns `code` (error reporting for entry points outside capi.cu).
int set_error(int code, const char* msg);

// Counts every kernel this library launches (for launch accounting).
void note_launches(unsigned n);
unsigned long long launches_so_far();

constexpr int kSweepThreads = 512;   // the sweep kernel's block size
constexpr int kAutotuneChoices = 9;  // layouts concord_autotune measures
constexpr int kPendCap = 8;          // pending row updates kept per row before a flush
constexpr int kDepth = 16;           // mailbox ring depth (a power of two, >= 4)

// Dynamic shared memory of the sweep kernel: pending lists of every owned
// row; the cluster variant adds its mailbox ring (kDepth x rows x value
// words) and per-row progress counters.
inline size_t sweep_dyn_smem(size_t elem, int row_warps, int rows_per_warp, bool cluster) {
  const size_t rows = (size_t)row_warps * rows_per_warp;
  size_t b = (elem + sizeof(int)) * rows * kPendCap;
  if (cluster) b += 8 * (elem / 4) * (size_t)kDepth * rows + 4 * rows;
  return b;
}

// Per-CTA partial results of the fused objective / KKT pass.
constexpr int kPartKkt = 0, kPartQuad = 1, kPartPen = 2, kPartLog = 3, kPartDelta = 4,
              kPartActive = 5, kPartBad = 6;
constexpr int kParts = 8;

// Final result block written by CTA 0.
constexpr int kResSweeps = 0, kResKkt = 1, kResObj = 2, kResDelta = 3, kResActive = 4,
              kResFirstDelta = 5, kResStatus = 6, kResRedo = 7,  // kResRedo: screened only
              kResPath = 8,  // screened path: index of the lambda a dense hand-over stopped at
              kResList = 9,  // screened: candidate list of the next sweep (-1: none valid)
              kResLazy = 10, // screened: sweeps that skipped the verification (lazy)
              kResAcc = 11,  // screened: accumulated lazy bound of the next sweep's list
              kResPartial = 12;  // screened: sweeps that verified only their loud rows' pairs
constexpr int kRes = 13;
constexpr int kHist = 4;  // per sweep: delta, kkt, objective, active pairs

// One problem of a batched launch of the sweep kernel: its own dimension,
// arrays, mailbox ring, barrier counter and range of CTAs.
template <typename T>
struct BatchProblem {
  int p, P, ld;
  int cta0, ctas;            // CTAs [cta0, cta0 + ctas) of the launch serve this problem
  T* W;                      // p x ld, W = Omega S
  T* Om;                     // p x ld, Omega
  const T* S;                // p x ld, S (padding columns zero)
  const T *sdiag, *sd1, *sd2;
  const double* sdiag64;     // s_ii in FP64
  double* omdiag64;          // FP64 diagonal of Omega (mixed precision only)
  unsigned long long* mbox;  // depth x (P+1) x words, tags below the launch's first
  unsigned* barrier;         // zeroed before the launch
  double* partials;          // ctas x kParts
  double* result;            // nk x kRes: the result of each lambda it walks
  float* cnt;                // nullable: slice k (p x p) += [w_ij != 0] after its lambda k
  int k0, nk;                // it walks lambdas[k0 .. k0 + nk)
  int stall_break;           // a lambda that ends on the stall rule ends the problem's walk
  int n_sweeps;              // > 0: its sweep limit per lambda (else the launch's)
};

template <typename T>
struct SweepArgs {
  int p, P, ld, rows_per_warp;
  int row_warps;              // warps per CTA that own rows (the rest join the KKT pass)
  T* W;                      // p x ld, W = Omega S
  T* Om;                     // p x ld, Omega (symmetric)
  const T* S;                // p x ld, S (padding columns zero)
  const T* sdiag;            // s_ii in T
  const T* sd1;              // sd1[v] = S[v][v-1] (v >= 1)
  const T* sd2;              // sd2[v] = S[v][next(v)], next(v) = v-2 cyclic on 1..P (0 if a bye)
  const double* sdiag64;     // s_ii in FP64
  double* omdiag64;          // FP64 diagonal of Omega (mixed precision only)
  unsigned long long* mbox;  // depth x (P+1) x words
  int depth;                 // must equal kDepth
  unsigned* barrier;         // zeroed before the launch
  WaitCtl wait;
  double* partials;          // gridDim.x x kParts
  double* hist;              // hist_len x kHist
  int hist_len;
  double* result;            // kRes
  double lambda, tol, delta_tol;
  int stop_rule, n_sweeps, kkt_only;
  int stall_stop;            // stop when the KKT residual stalls (FP32 phase)
  unsigned poll_ns;          // back-off between mailbox polls (0: none)
  unsigned tag_base;
  int fault_vertex, fault_step;
  // batched launch (launch_sweep_batch): problems and the lambda path every
  // problem walks (warm-started, n_sweeps sweeps at most per lambda)
  const BatchProblem<T>* probs;
  int n_probs;
  const double* lambdas;
  int n_lambda;
  float* batch_cnt;          // (set per problem inside the kernel) its support counts
  int stall_break;           // (set per problem inside the kernel)
};

// cluster = true: the whole grid is one thread-block cluster (grid <= 16).
cudaError_t launch_sweep(const SweepArgs<double>& a, int grid, int block, bool cluster,
                         cudaStream_t st);
cudaError_t launch_sweep(const SweepArgs<float>& a, int grid, int block, bool cluster,
                         cudaStream_t st);
cudaError_t sweep_occupancy(bool mixed, int block, int* blocks_per_sm);
// Batched launch: a.probs[0..n_probs) with their CTA ranges covering
// [0, grid); each problem runs the lambda path a.lambdas[0..n_lambda) from
// its current iterate, stopping each lambda on a.stop_rule / a.tol, on the
// FP32 stall rule (stall_stop) or after a.n_sweeps sweeps, and writes one
// result row per lambda.  Problems are independent: they share the launch,
// the abort word and nothing else.
cudaError_t launch_sweep_batch(const SweepArgs<double>& a, int grid, int block, cudaStream_t st);
cudaError_t launch_sweep_batch(const SweepArgs<float>& a, int grid, int block, cudaStream_t st);
// Largest launchable cluster (power of two <= 16; 0 if none).
cudaError_t sweep_cluster_size(bool mixed, int block, int row_warps, int rows_per_warp, int* cs);

// ---- screened sweep (screened.cu)
// One persistent cooperative launch of Algorithm 1's outer iterations that
// visits only the candidate pairs of each sweep (the pairs that can change)
// and verifies every other pair afterwards; see screened.cu.
constexpr int kScreenThreads = 512;
constexpr int kRowList = 64;      // changes of one row staged per warp in the row pass
constexpr int kCtrCand = 0;       // ctr[0], ctr[1]: lengths of the two candidate lists
constexpr int kCtrFail = 2;       // failing pairs found by the verification
constexpr int kCtrTerms = 3;      // correction terms of the current candidate set
constexpr int kCtrJacDone = 5;    // the fixed-point iteration settled
constexpr int kCtrTermsPred = 6;  // correction terms the current list needs (sum over rows of k (k - 1) / 2)
constexpr int kCtrLoud = 7;       // rows whose lazy bound left half the margin this sweep
constexpr int kCtrs = 8;
constexpr int kJacMax = 64;       // fixed-point iterations of the chain before the dense kernel takes the sweep
constexpr int kLoudMax = 256;     // rows a partial verification takes (more: a full sweep)
constexpr int kStatusDense = 5;   // result status: the next sweep needs the dense kernel
constexpr int kPendRow = 32;      // deferred W updates a row holds (lazy sweeps)

template <typename T>
struct ScreenWork {
  int* ctr;                 // kCtrs counters (zeroed before the launch)
  int2* cand[2];            // candidate pairs (i < j): current sweep / next sweep; a
                            // candidate's number is its position in the list
  int* cnt_r[2];            // [p + 1] candidates per row of each list (counted at the push)
  int2* fail;               // non-candidate pairs that failed the verification
  int *off_r, *cur_r;       // [p + 1] row buckets of the current list: offsets, cursors
  int *nd_pi, *nd_pj;       // position of each candidate in the lists of rows i and j
  int* row_ent;             // [2 nc_cap] candidates of each row, in colour-step order
  int* term_ptr;            // [nc_cap + 1] first correction term of each candidate
  int* term_pred;           // [term_cap] earlier candidate whose change the term carries
  T* term_s;                // [term_cap] the S entry it multiplies
  T* nd_rec;                // [4 nc_cap] per candidate: W_ij, W_ji, w_ij at the sweep start, s_ii + s_jj
  T *nd_delta, *nd_new;     // change and new value of each candidate
  T* nd_d2;                 // [nc_cap] second buffer of the fixed-point iteration
  unsigned long long* jac;  // [kJacMax] per fixed-point round: arrivals + (CTAs whose changes moved) << 32
  T* diag_old;              // [p] diagonal before the sweep (for a redo)
  double* omdiag_old;       // [p] FP64 diagonal before the sweep (mixed precision)
  double* diag_new;         // [p] the sweep's new FP64 diagonal, committed after the row pass
  double* dpart;            // [grid] per-CTA largest row bound of the sweep (lazy verification)
  int* dfill;               // [grid] per-CTA largest pending-list fill the sweep would need
  // deferred row updates of lazy sweeps: row i's true W is its stored row with
  // pend (u, d) applied in order, w <- d S_u + w; pend_n[i] entries are valid,
  // the slots up to pend_new[i] hold the current sweep's tentative ones
  T* diag_dd;               // [p] the sweep's diagonal change in T (W_i += dd S_i)
  int* pend_u;              // [p x kPendRow]
  T* pend_d;                // [p x kPendRow]
  int *pend_n, *pend_new;   // [p] (zeroed before the launch)
  // per-row lazy bound: rowacc[i] bounds how far G_ij of a pair outside the
  // list has moved since row i's pairs were screened (through row i's
  // changes); rowa_new is rowacc + this sweep's D_i, loudf marks the rows
  // whose rowa_new exceeds half the margin (listed in loud when they fit)
  double* rowacc;           // [p]
  double* rowa_new;         // [p]
  double* apart;            // [grid] per-CTA largest rowa_new of the quiet rows
  int* loud;                // [kLoudMax]
  int* loudf;               // [p]
  int nc_cap, term_cap, fail_cap;
};

template <typename T>
struct ScreenArgs {
  int p, P, ld;
  T* W;                     // p x ld, W = Omega S (in and out)
  T* Wb;                    // p x ld scratch: W after the sweep
  T* V;                     // p x ld scratch: W_ij when pair (i, j) is visited (NaN: candidate)
  T* Om;                    // p x ld, Omega
  const T* S;               // p x ld, S (padding columns zero)
  const T* sdiag;           // s_ii in T
  const double* sdiag64;    // s_ii in FP64
  double* omdiag64;         // FP64 diagonal of Omega (mixed precision only)
  ScreenWork<T> w;
  unsigned* barrier;        // zeroed before the launch
  WaitCtl wait;
  double* partials;         // gridDim.x x kParts
  double* hist;             // hist_len x kHist
  int hist_len;
  double* result;           // kRes
  double lambda, tol, delta_tol;
  int stop_rule, n_sweeps, kkt_only, stall_stop;
  int max_redo;             // verification rounds per sweep before giving up (status 5)
  int start_list;           // >= 0: the first sweep uses candidate list start_list as the
                            // previous launch left it (counts, row offsets, term count);
                            // -1: screen the starting point
  int start_scan;           // with start_list: only its counts are in place (a list
                            // screened outside the kernel); the first build scans them
  const int* input_flag;    // nullable: nonzero when a check of the input failed (the
                            // launch then ends before its first sweep, status 2)
  // lambda path (path_n > 0): lambdas path_lambda[path_start .. path_n), each
  // swept until its stopping rule, warm-started from the previous one
  const double* path_lambda;
  int path_n, path_start;
  double* path_res;         // [path_n x kRes] result of each lambda
  T* path_om;               // nullable: Omega after each lambda, slice k at k p ldo
  int path_ldo;
  float* path_cnt;          // nullable: slice k (p x p) += [w_ij != 0] after lambda k (atomic)
  // lazy verification: a sweep whose changes provably keep every pair outside
  // the candidates below the threshold skips the verification pass and keeps
  // its candidate list (and the build of it) for the next sweep
  const float* mrow;        // [p] m[u] >= max_{x != u} |s_ux|
  int lazy_verify;
  int keep_w;               // 1: W is left up to date at the end; 0: deferred updates may
                            // be dropped (the host rebuilds W from Omega before using it)
  int path_break_stall;     // a lambda that ends on the stall rule ends the launch (the
                            // host polishes it in FP64 and resumes the path after it)
};

size_t screened_dyn_smem(bool mixed);
cudaError_t launch_screened(const ScreenArgs<double>& a, int grid, cudaStream_t st);
cudaError_t launch_screened(const ScreenArgs<float>& a, int grid, cudaStream_t st);
cudaError_t screened_occupancy(bool mixed, int* blocks_per_sm);

cudaError_t launch_refresh_w(const double* Om, const double* S, double* W, int p, int ld, int sms,
                             cudaStream_t st);

// ---- data preparation and Gram (prep_gram.cu)
// Column statistics of X (n x p, row stride ldx): mean[i] and inv_scale[i]
// per `prep` (0: mean 0, scale 1; 1: centre; 2: centre and 1/sd, population
// variance).  bad (int) is set to 1 if a column is constant under prep 2 or
// non-finite.
cudaError_t launch_col_stats(const void* X, int x_f32, int n, int p, int ldx, int prep,
                             double* mean, double* inv_scale, int* bad, cudaStream_t st);
// Z = (X - mean) * inv_scale into Z (n x ldz, type z_f32 ? float : double);
// columns p..ldz-1 are zero.
cudaError_t launch_apply_prep(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, void* Z, int z_f32, int ldz,
                              cudaStream_t st);
// S = Z^T Z * scale on CUDA cores (upper-triangle tiles, mirrored).
cudaError_t launch_syrk_f64(const double* Z, int n, int p, int ldz, double* S, int lds, double scale,
                            cudaStream_t st);
cudaError_t launch_syrk_f32(const float* Z, int n, int p, int ldz, float* S, int lds, float scale,
                            cudaStream_t st);

// ---- small utilities (util.cu)
// out[r*ldo + c] = (To) in[r*ldi + c] for r < rows, c < cols; zero for cols <= c < ldo.
cudaError_t launch_convert(const void* in, int in_f32, int ldi, void* out, int out_f32, int ldo,
                           int rows, int cols, cudaStream_t st);
// d64[i] = A[i*lda+i]; dT[i] (type t_f32) likewise; bad |= 1 if not > 0, 2 if non-finite.
cudaError_t launch_extract_diag(const void* A, int a_f32, int lda, int p, double* d64, void* dT,
                                int t_f32, int* bad, cudaStream_t st);
// Sub-diagonal vectors of the circle-method walk: sd1[v] = S[v][v-1] and
// sd2[v] = S[v][v-2] for v >= 3, S[1][P-1], S[2][P] (0 where the column is the
// extra vertex of odd p); entry 0 is 0.
cudaError_t launch_subdiag(const void* S, int s_f32, int ld, int p, int P, void* sd1, void* sd2,
                           cudaStream_t st);
// a[0..n) = v.
cudaError_t launch_fill_f64(double* a, double v, int n, cudaStream_t st);
// m[u] >= max_{x != u} |S[u][x]| (float, rounded up; for FP32 S one step
// above, so it also bounds an FP64 copy of S rounded to this S).
cudaError_t launch_row_absmax(const void* S, int s_f32, int ld, int p, float* m, cudaStream_t st);
// A (p x ld, type) = identity with zero padding.
cudaError_t launch_set_identity(void* A, int a_f32, int p, int ld, cudaStream_t st);
// Mixed-precision start after a Gram into the FP32 S (p x ld, zero padding),
// in one pass over S: W = S, Omega = I, S64 = S widened, m[u] as
// launch_row_absmax, the diagonal (FP64 and FP32; bad |= 8 if non-finite,
// 16 if not > 0), the walk vectors of launch_subdiag in both precisions, and
// the FP64 diagonal of Omega = 1.
struct ResetMixedArgs {
  const float* S;
  int ld, p, P;
  float *W, *Om;
  double* S64;
  float* mrow;
  double* sdiag64;
  float* sdiag32;
  float *sd1, *sd2;
  double *sd1_64, *sd2_64;
  double* omdiag64;
  int* bad;
  // optional screen of the starting point (Omega = I, W = S) for one lambda:
  // pairs i < j with |(0 - s_ij) - s_ji| > lam_s join cand, as the screened
  // kernel's own start screen would push them (lam_s <= 0: no screen)
  float lam_s;
  int2* cand;
  int* n_cand;
  int* cnt_r;
  int nc_cap;
};
cudaError_t launch_reset_mixed(const ResetMixedArgs& a, cudaStream_t st);
// bad |= 1 if |A - A^T| != 0 anywhere or a non-finite entry is met.
cudaError_t launch_check_symmetric(const void* A, int a_f32, int p, int lda, int* bad,
                                   cudaStream_t st);
// out (FP64 bits as u64, must start at 0) = max_{i<j} |s_ij| (s_ii^-1/2 + s_jj^-1/2).
cudaError_t launch_lambda_max(const double* S, int p, int ld, unsigned long long* out,
                              cudaStream_t st);

// ---- lambda path and stability selection helpers (util.cu)
// out (nr x p, FP64, dense) = rows `rows` of X (row stride ldx).
cudaError_t launch_gather_rows(const void* X, int x_f32, int ldx, const int* rows, int nr, int p,
                               double* out, cudaStream_t st);
// cnt[r * p + c] += 1 (atomically) where Om[r * ld + c] != 0.
cudaError_t launch_support_add(const void* Om, int f32, int ld, int p, float* cnt, cudaStream_t st);
cudaError_t launch_scale_f32(float* a, size_t n, float s, cudaStream_t st);

// ---- tensor-core Gram (gram_tc.cu)
// Splits each standardized element into tf32 hi + lo and writes them
// transposed: Zt_hi / Zt_lo are p_pad x n_pad (K-major), zero padded.  With
// zt (nullable) the FP32 value itself is also written transposed
// (p_pad x ldz, ldz <= n_pad); hi / lo may be NULL when zt is given.
cudaError_t launch_split_tf32(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, float* zt_hi, float* zt_lo, int n_pad,
                              int p_pad, cudaStream_t st, float* zt = nullptr, int ldz = 0);
// S (p x lds, FP32) = (hi hi^T + hi lo^T + lo hi^T) * scale with tcgen05.mma
// kind::tf32 (n_pad a multiple of 32, p_pad of 128).  A device-side wait that
// runs out sets bit 4 of *status.  cudaErrorNotSupported if not sm_103.
cudaError_t launch_gram_tf32x3(const float* zt_hi, const float* zt_lo, int n_pad, int p_pad, int p,
                               float* S, int lds, float scale, int* status, cudaStream_t st);
// The same split into bf16 hi + lo (raw 16-bit patterns, p_pad x n_pad,
// n_pad a multiple of 64) and the Gram with tcgen05.mma kind::f16 (3xBF16).
cudaError_t launch_split_bf16(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, uint16_t* zt_hi, uint16_t* zt_lo, int n_pad,
                              int p_pad, cudaStream_t st, float* zt = nullptr, int ldz = 0);

// ---- FP64-accurate S on the solution's neighbourhood (refine.cu)
// Pairs collected from a dense iterate: w_ij != 0 or |G_ij| > (1 - margin)
// lambda (the screen's margin).
constexpr double kRefineMargin = 0.1;
constexpr int kRefineDone = 0;     // ctr: entries recomputed
constexpr int kRefineOwn = 1;      // ctr: length of the collected list (no candidate list given)
constexpr int kRefineDropped = 2;  // ctr: collected pairs that did not fit
constexpr int kRefineDs = 3;       // ctr: float bits of max |new - old| over recomputed entries
constexpr int kRefineCtrs = 4;
struct RefineArgs {
  int p, ld, n, ldn, sms;
  const float* zt;           // p_pad x ldn: standardized data in FP32, transposed
  const int2* cand;          // candidate pairs (i < j) of the next sweep, or NULL
  const int* n_cand;         // device: their number
  const float *Om32, *W32;   // the FP32 iterate (to collect pairs when cand is NULL)
  float thr;                 // collection threshold on |W_ij + W_ji|
  int2* own_cand;            // [own_cap] collected pairs
  int own_cap;
  double* S64;               // p x ld: entries recomputed in place (both triangles)
  float* S32;                // p x ld: the same entries rounded to FP32
  float* mrow;               // [p] row bounds max_{x != u} |s_ux|, raised where an entry grows
  int *nbr_cnt, *nbr_off, *nbr_cur;  // [p + 1]
  int* nbr;                  // [2 x max(list length)]
  unsigned* bitmap;          // [refine_bitmap_words(p)]
  int* ctr;                  // [kRefineCtrs]
};
size_t refine_bitmap_words(int p);

// Screening margin: a pair is a candidate of the next sweep when its value is
// nonzero or |G_ij| > (1 - kScreenMargin) lambda at the sweep's start.  Any
// superset of the pairs that change gives the same iterates (a candidate
// that stays below the threshold gets a zero change); the margin catches the
// pairs that cross the threshold during the sweep, which would otherwise
// fail the verification and force a redo of the sweep.
constexpr double kScreenMargin = 0.1;

// Lazy verification.  Every pair outside the candidate list had
// |G_ij| <= (1 - kScreenMargin) lambda when the list was screened.  A change d
// of a candidate (i, u) moves W_ix by d s_ux for x != u, so by at most
// |d| m_u (m_u = max_{x != u} |s_ux|), and a diagonal change moves W_ix by at
// most |dw| m_i.  With D_i the sum of those bounds over a sweep's changes of
// row i, G_ij of a pair outside the list moves by at most D_i + D_j <=
// 2 max_i D_i per sweep.  While the bounds accumulated since the screen stay
// within (kScreenMargin - kLazySlack) lambda, no such pair can reach the
// threshold at its visit (so the verification would pass) nor at the sweep's
// end (so its KKT term is zero): the sweep skips the verification pass, and
// the list, with its build, serves the next sweep too.  kLazySlack lambda is
// left for rounding (far more than FP32 accumulates on W over a few sweeps).
constexpr double kLazySlack = 0.01;

// ---- sparse FP64 polish (polish.cu).  FP64 sweeps of a mixed solve that
// keep every pair outside the FP32 phase's candidate list at zero (the lazy
// verification bound, carried over with the FP32 -> FP64 change of S): each
// W entry a sweep reads is formed from the nonzeros of Omega and S, so W is
// never materialised.
constexpr int kStatusNeedW = 6;       // result status: the bound failed; W must be rebuilt
constexpr int kStatusCapacity = 7;    // result status: the terms did not fit (ctr holds the need)
constexpr int kPolishThreads = 512;
constexpr int kPolishMaxRounds = 1024;  // fixed-point rounds per sweep before giving up
constexpr int kPolOverflow = 3;       // ctr: terms needed when they do not fit (0: fit)
constexpr int kPolSMax = 6;           // ctr[6..7]: max |s_ux| (double bits)
constexpr int kPolLoud = 8;           // ctr: rows whose bound leaves half the margin this sweep
constexpr int kPolFail = 9;           // ctr: a verified pair would have left zero
constexpr int kPolCtrs = 10;
constexpr int kPolLoudMax = 256;      // rows one polish sweep verifies (more: W is rebuilt)
struct PolishWork {
  int* ctr;          // [kPolCtrs] (zeroed before the launch)
  unsigned long long* rslot;  // [3] the fixed-point rounds' arrivals and flags, in turn (zeroed)
  int* deg;          // [p + 1] entries per row (zeroed before the launch)
  int* off;          // [p + 1] row offsets of the entries
  int* toff;         // [p + 1] row offsets of the terms (deg (deg - 1) per row)
  int* cur;          // [p] fill cursors
  int* ent0;         // [2 nc_cap] row entries (candidate numbers) as filled
  int* ent;          // [2 nc_cap] row entries in colour-step order
  int* pos;          // [2 nc_cap] rank of candidate k in row i (2k) and in row j (2k + 1)
  int* term_q;       // [term_cap] candidate of each term
  double* term_s;    // [term_cap] the S entry it multiplies
  double* om;        // [nc_cap] value of each candidate
  double* den;       // [nc_cap] s_ii + s_jj
  double* base;      // [2 nc_cap] W_ij - omega_ij s_jj (2k) and W_ji - omega_ij s_ii (2k + 1)
  double* d0;        // [nc_cap] fixed-point iterates of the changes
  double* d1;        // [nc_cap]
  double* nw;        // [nc_cap] new value of each candidate
  double* diag;      // [p] the diagonal of Omega
  double* diag_new;  // [p]
  double* dpart;     // [grid] per-CTA largest row bound of a sweep
  // per-row bound on how far G_ij of a pair outside the list has moved since
  // the screen (pair bound rowa_i + rowa_j); rows beyond half the margin are
  // verified exactly (their W entries are short sums over Omega's nonzeros)
  double* rowa;      // [p]
  double* rowb;      // [p] rowa + this sweep's D_i
  int* loud;         // [kPolLoudMax]
  int* loudf;        // [p] 0: quiet; 2: loud, its pairs within 0.9 lambda; 1: loud, some beyond
  int nc_cap, term_cap;
};
struct PolishArgs {
  int p, P, ld;
  double* Om;              // p x ld FP64 Omega (zeroed): the result, diagonal included
  const float* Om32;       // p x ld FP32 Omega of the FP32 phase (its off-diagonal values)
  const double* omdiag;    // [p] its FP64 diagonal
  const double* S;         // p x ld FP64 S
  const double* sdiag;     // [p] s_ii
  const float* mrow;       // [p] m[u] >= max_{x != u} |s_ux|
  const int2* cand;        // candidate pairs (i < j) left by the FP32 phase
  const int* n_cand;       // device: their number
  const int* ds_bits;      // nullable: float bits of max |S64 - S32 used by the FP32 phase|
  double acc0;             // lazy bound accumulated by the FP32 phase since its screen
  const double* rowacc;    // nullable: the FP32 phase's per-row bound (pair bound a_i + a_j);
                           // without it every row starts at acc0 / 2
  PolishWork w;
  unsigned* barrier;       // zeroed before the launch
  WaitCtl wait;
  double* partials;        // grid x kParts
  double* hist;
  int hist_len;
  double* result;          // kRes
  double lambda, tol, delta_tol;
  int stop_rule, n_sweeps;
};
cudaError_t launch_polish(const PolishArgs& a, int grid, cudaStream_t st);
cudaError_t launch_refine_s(const RefineArgs& a, cudaStream_t st);
cudaError_t launch_gram_bf16x3(const uint16_t* zt_hi, const uint16_t* zt_lo, int n_pad, int p_pad,
                               int p, float* S, int lds, float scale, int* status, cudaStream_t st);

}  // namespace concord
