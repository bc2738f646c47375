// Host side of the C ABI declared in include/concord.h.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <thread>
#include <vector>

#include "concord.h"
#include "adjoint.h"
#include "prep_stats.h"
#include "kernels.h"

using namespace concord;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(expr)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      if (e_ == cudaErrorMemoryAllocation)                                               \
        return fail(CONCORD_E_NOMEM, "%s: %s", #expr, cudaGetErrorString(e_));           \
      if (e_ == cudaErrorCooperativeLaunchTooLarge)                                      \
        return fail(CONCORD_E_OCCUPANCY, "%s: %s", #expr, cudaGetErrorString(e_));       \
      return fail(CONCORD_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));              \
    }                                                                                    \
  } while (0)

constexpr int kMailboxDepth = kDepth;
constexpr int kHistCap = 8192;
constexpr int kMaxTimedLaunches = 16;
constexpr int kDefaultPollNs = 0;

int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

int concord::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct concord_state {
  int device = -1, sms = 0;
  int p = 0, pe = 0, P = 0, ld = 0, precision = 0, n_cap = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  // working set: float for CONCORD_MIXED, double for CONCORD_FP64
  void *S = nullptr, *W = nullptr, *Om = nullptr, *sdiagT = nullptr;
  double* sdiag64 = nullptr;
  double* omdiag64 = nullptr;  // mixed only
  float* mrow = nullptr;       // [p] m[u] >= max_{x != u} |s_ux| (lazy verification bound)
  bool lazy_verify = true;
  bool screen_keep_w = true;   // one-shot: false lets the next screened launch drop deferred W updates
  void *sd1 = nullptr, *sd2 = nullptr;    // sub-diagonal walk vectors, working precision
  double *sd1_64 = nullptr, *sd2_64 = nullptr;  // FP64 versions (mixed polish)
  // FP64 copies (mixed) or aliases of the working set (fp64)
  double *S64 = nullptr, *W64 = nullptr, *Om64 = nullptr;
  bool om64_current = false;  // mixed: FP64 copies hold the latest iterate
  int start_list = -1;        // one-shot: the next screened launch starts from this list
  bool start_scan = false;    // one-shot, with start_list: the list's row offsets still to scan
  // a start screen made with the one-pass start (list 0, for prescreen_lambda):
  // the next mixed run at that lambda starts from it
  bool prescreen = false;
  double prescreen_lambda = 0.0;
  // the Gram's and the one-pass start's checks (flag) not read yet: the next
  // screened launch reads the word on the device and the host after it
  bool flag_pending = false;
  unsigned long long* mbox = nullptr;
  int depth = kMailboxDepth;
  unsigned* barrier = nullptr;
  int* abort_info = nullptr;  // [0] abort word, [1] vertex, [2] step
  double* partials = nullptr;
  double* hist = nullptr;
  double* result = nullptr;
  int* flag = nullptr;
  unsigned long long* lmax = nullptr;
  unsigned tag_base = 1;
  double timeout_s = 2.0;
  int fault_vertex = -1, fault_step = -1;
  int max_grid = 0;
  int hist_rows = 0;
  // data workspace
  double *mean = nullptr, *inv_scale = nullptr;
  void* Z = nullptr;
  int ldz = 0;
  double* Xstage = nullptr;  // n_cap x p FP64, host-data path
  float *zt_hi = nullptr, *zt_lo = nullptr;
  int n_pad = 0, p_pad = 0;
  // mixed: the standardized data in FP32, transposed (p_pad x zt_ldn), kept
  // for the FP64-accurate S entries recomputed before a polish
  float* zt32 = nullptr;
  int zt_ldn = 0, zt_n = 0;
  bool zt_valid = false;  // zt32 holds the data S came from
  bool refine = true;     // recompute the neighbourhood's S entries before a polish
  struct {
    int *cnt = nullptr, *off = nullptr, *cur = nullptr, *nbr = nullptr, *ctr = nullptr;
    int2* cand = nullptr;
    unsigned* bitmap = nullptr;
    int nbr_cap = 0, cand_cap = 0;
  } rf;
  int* h_rf = nullptr;  // pinned: entries recomputed by the last promotion
  // sparse FP64 polish (polish.cu): one device block carved into its arrays
  struct {
    void* mem = nullptr;
    int nc_cap = 0, term_cap = 0;
    PolishWork w;
  } pol;
  bool sparse_polish = true;  // mixed: polish on the candidates without rebuilding W
  bool w64_stale = false;     // mixed: W64 does not hold Omega64 S64 (after a sparse polish)
  int gram_mode = CONCORD_GRAM_FP64;
  int rows_per_warp = 0;  // 0: automatic (one row per lane)
  int sweep_variant = 0;  // 0 auto, 1 grid, 2 cluster (CONCORD_SWEEP_*)
  int poll_ns = -1;       // back-off between mailbox polls (-1: default)
  int cluster_size = -1;  // largest launchable cluster (-1: not queried yet)
  int last_variant = 0;
  // screened-sweep scratch (allocated on first use): W after the sweep, W at
  // each pair's visit, candidate lists and per-candidate work arrays
  void *Wb = nullptr, *V = nullptr, *scr = nullptr;
  int nc_cap = 0, term_cap = 0;
  int screened_grid = 0;
  int max_ctas = 0;  // > 0: persistent launches use at most this many CTAs (concurrent workers)
  int last_batch_rows = 0;  // rows per warp the last batched stability run used
  bool path_polish = true;  // mixed paths: FP64 polish of a lambda whose FP32 sweeps stall
  // lambda path / stability selection buffers (allocated on demand)
  double *path_lam = nullptr, *path_res = nullptr;
  int path_cap = 0;
  int* rows_dev = nullptr;
  size_t rows_cap = 0;
  // implicit differentiation (allocated on demand): CSR of the active set,
  // the iteration vectors on its entries, and the data-gradient workspace
  // CSR readout of Omega (allocated on demand)
  int *csr_cnt = nullptr, *csr_rowptr = nullptr, *csr_col = nullptr, *csr_row = nullptr;
  double* csr_val = nullptr;
  int csr_cap = 0;
  struct {
    int nnz = 0, cap = 0;
    int *cnt = nullptr, *rowptr = nullptr, *bad = nullptr;
    int *col = nullptr, *erow = nullptr, *mirror = nullptr;
    double *om = nullptr, *minv = nullptr, *b = nullptr, *x = nullptr, *r = nullptr;
    double *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
    double *scal = nullptr;  // [kAdjRes] CG results, then the held-out loss
    bool rhs_ready = false, solved = false;
    int n_cap = 0;           // rows of the data workspace
    double *Z = nullptr, *P = nullptr, *Q = nullptr, *dZ = nullptr;
    double *part1 = nullptr, *part2 = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *mean = nullptr, *scale = nullptr;
  } adj;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t lev[2 * kMaxTimedLaunches] = {};
  double launch_ms[kMaxTimedLaunches] = {};
  int launch_sweeps[kMaxTimedLaunches] = {};
  int n_launch = 0;
  // pinned host mirrors
  double* h_result = nullptr;
  int* h_abort = nullptr;
  int* h_flag = nullptr;
};

namespace {

bool is_mixed(const concord_state* st) { return st->precision == CONCORD_MIXED; }

int check_state(concord_state* st) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  CK(cudaSetDevice(st->device));
  return CONCORD_OK;
}

// The errors behind the bits of the data checks (Gram: 1 constant column,
// 2 non-finite entry, 4 device wait ran out; one-pass start: 8 non-finite
// diagonal, 16 diagonal <= 0).
int input_flag_error(int bad) {
  if (bad & 4) return fail(CONCORD_E_TIMEOUT, "tensor-core Gram: a device-side wait ran out");
  if (bad & 2) return fail(CONCORD_E_NONFINITE, "X has a non-finite entry");
  if (bad & 1) return fail(CONCORD_E_NONPOS_DIAG, "X has a constant column");
  if (bad & 8) return fail(CONCORD_E_NONFINITE, "S has a non-finite diagonal entry");
  if (bad & 16) return fail(CONCORD_E_NONPOS_DIAG, "S has a diagonal entry <= 0 (constant column?)");
  return CONCORD_OK;
}

int read_flag(concord_state* st, int* out) {
  CK(cudaMemcpyAsync(st->h_flag, st->flag, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  *out = *st->h_flag;
  return CONCORD_OK;
}

struct RunOut {
  int status = CONCORD_OK;
  int sweeps = 0, first_delta = 0;
  double kkt = 0, obj = 0, delta = 0, active = 0;
  int to_vertex = -1, to_step = -1;
  bool stalled = false;
  int redos = 0, dense_sweeps = 0;  // screened runs
  int next_list = -1;               // screened: candidate list left for the next sweep
  int s_refined = 0;                // S entries recomputed before the polish
  double acc = 0;                   // screened: lazy bound accumulated on the next sweep's list
  int lazy = 0;                     // screened sweeps that skipped the verification
  int sparse = 0;                   // polish sweeps run by the sparse polish
  int partial = 0;                  // screened sweeps that verified only their loud rows
};

// One persistent launch: n_sweeps outer iterations (fewer if the stopping
// rule holds first), or only the objective / KKT pass when kkt_only.
template <typename T>
int launch_dense(concord_state* st, T* S, T* W, T* Om, const T* sdiagT, double* omdiag64,
                 double lambda, double tol, int stop_rule, int n_sweeps, int kkt_only,
                 int hist_offset, int stall_stop, RunOut* out, bool bandwidth = false) {
  const int p = st->p;
  const bool mixed = sizeof(T) == 4;
  // `row_warps` warps of each CTA own rows (one row per lane, up to `R` rows
  // per warp); every warp takes part in the objective / KKT pass.
  const int block = kSweepThreads;
  // AUTO: FP32 sweeps take the cluster variant (lowest exchange latency);
  // FP64 sweeps the grid variant, which spreads the FP64 arithmetic over
  // every SM.  Rows per warp: 32 in a cluster, 8 on the grid.  Explicit
  // settings apply to sweeps in the state's working precision; the FP64
  // polishing sweeps of a mixed state keep the FP64 defaults.
  const bool own = mixed == is_mixed(st);
  const bool layout_set = own && (st->sweep_variant == CONCORD_SWEEP_GRID ||
                                  st->sweep_variant == CONCORD_SWEEP_CLUSTER);
  // bandwidth: sweeps handed over by the screened kernel change most pairs;
  // they take the grid layout with one row per warp (all SMs stream rows)
  const int variant = bandwidth    ? CONCORD_SWEEP_GRID
                      : layout_set ? st->sweep_variant
                                   : (mixed ? CONCORD_SWEEP_CLUSTER : CONCORD_SWEEP_GRID);
  bool cluster = false;
  int grid = 0, row_warps = 0, R = 0;
  int want = bandwidth ? 1 : (own && st->rows_per_warp > 0) ? st->rows_per_warp : 32;
  if (variant != CONCORD_SWEEP_GRID) {
    if (st->cluster_size < 0) {
      int cs = 0;
      CK(sweep_cluster_size(mixed, block, block / 32, 32, &cs));
      st->cluster_size = cs;
    }
    const int cs = st->cluster_size;
    if (cs >= 2 && (long long)cs * (block / 32) * 32 >= p) {
      cluster = true;
      grid = cs;
      row_warps = (p + want * cs - 1) / (want * cs);
      if (row_warps < 1) row_warps = 1;
      if (row_warps > block / 32) row_warps = block / 32;
      R = (p + cs * row_warps - 1) / (cs * row_warps);
    } else if (variant == CONCORD_SWEEP_CLUSTER && own && st->sweep_variant == CONCORD_SWEEP_CLUSTER) {
      return fail(CONCORD_E_ARG, "p=%d does not fit one cluster of %d CTAs", p, cs);
    }
  }
  if (!cluster) {
    if (!bandwidth && !(own && st->rows_per_warp > 0)) want = 8;
    int occ = 0;
    CK(sweep_occupancy(mixed, block, &occ));
    if (occ < 1)
      return fail(CONCORD_E_OCCUPANCY, "sweep kernel cannot run %d threads per block", block);
    grid = st->sms * occ;
    const int need = (p + 31) / 32;
    if (grid > need) grid = need;
    if (grid > st->max_grid) grid = st->max_grid;
    if (st->max_ctas > 0 && grid > st->max_ctas) grid = st->max_ctas;
    row_warps = (p + want * grid - 1) / (want * grid);
    if (row_warps < 1) row_warps = 1;
    if (row_warps > block / 32) row_warps = block / 32;
    const int TW = grid * row_warps;
    R = (p + TW - 1) / TW;
  }
  if (R > 32) return fail(CONCORD_E_ARG, "p=%d needs %d rows per warp (max 32)", p, R);
  st->last_variant = cluster ? CONCORD_SWEEP_CLUSTER : CONCORD_SWEEP_GRID;

  // keep step tags monotone over the state's lifetime; restart them (and
  // clear the mailboxes) well before 32-bit overflow
  const unsigned long long span = (unsigned long long)(n_sweeps + 1) * (unsigned)st->P + st->depth;
  if ((unsigned long long)st->tag_base + span >= (1ull << 31)) {
    CK(cudaMemsetAsync(st->mbox, 0, sizeof(unsigned long long) * 2 * (size_t)st->depth * st->pe,
                       st->stream));
    st->tag_base = 1;
  }
  CK(cudaMemsetAsync(st->barrier, 0, sizeof(unsigned), st->stream));
  CK(cudaMemsetAsync(st->abort_info, 0, 3 * sizeof(int), st->stream));

  SweepArgs<T> a;
  memset(&a, 0, sizeof a);
  a.p = p;
  a.P = st->P;
  a.ld = st->ld;
  a.rows_per_warp = R;
  a.row_warps = row_warps;
  a.stall_stop = stall_stop;
  a.poll_ns = (unsigned)(st->poll_ns >= 0 ? st->poll_ns : kDefaultPollNs);
  a.W = W;
  a.Om = Om;
  a.S = S;
  a.sdiag = sdiagT;
  if (sizeof(T) == 4) {
    a.sd1 = (const T*)st->sd1;
    a.sd2 = (const T*)st->sd2;
  } else {
    a.sd1 = (const T*)st->sd1_64;
    a.sd2 = (const T*)st->sd2_64;
  }
  a.sdiag64 = st->sdiag64;
  a.omdiag64 = omdiag64;
  a.mbox = st->mbox;
  a.depth = st->depth;
  a.barrier = st->barrier;
  a.wait.abort = st->abort_info;
  a.wait.info = st->abort_info + 1;
  a.wait.timeout_ns = (uint64_t)(st->timeout_s * 1e9);
  a.partials = st->partials;
  a.hist = st->hist + (size_t)hist_offset * kHist;
  a.hist_len = kHistCap - hist_offset;
  a.result = st->result;
  a.lambda = lambda;
  a.tol = tol;
  a.delta_tol = 1e-5;
  a.stop_rule = stop_rule;
  a.n_sweeps = n_sweeps;
  a.kkt_only = kkt_only;
  a.tag_base = st->tag_base;
  a.fault_vertex = st->fault_vertex;
  a.fault_step = st->fault_step;
  st->fault_vertex = -1;  // one-shot
  st->fault_step = -1;

  const int slot_ev = st->n_launch < kMaxTimedLaunches ? st->n_launch : -1;
  if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev], st->stream));
  CK(launch_sweep(a, grid, block, cluster, st->stream));
  if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev + 1], st->stream));
  st->tag_base += (unsigned)span;

  CK(cudaMemcpyAsync(st->h_result, st->result, kRes * sizeof(double), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaMemcpyAsync(st->h_abort, st->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  const double* r = st->h_result;
  out->sweeps = (int)r[kResSweeps];
  out->kkt = r[kResKkt];
  out->obj = r[kResObj];
  out->delta = r[kResDelta];
  out->active = r[kResActive];
  out->first_delta = (int)r[kResFirstDelta];
  if (slot_ev >= 0) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, st->lev[2 * slot_ev], st->lev[2 * slot_ev + 1]));
    st->launch_ms[slot_ev] = ms;
    st->launch_sweeps[slot_ev] = out->sweeps;
    st->n_launch = slot_ev + 1;
  }
  const int code = (int)r[kResStatus];
  if (st->h_abort[0] != 0) {
    out->status = CONCORD_E_TIMEOUT;
    out->to_vertex = st->h_abort[1];
    out->to_step = st->h_abort[2];
    return fail(CONCORD_E_TIMEOUT, "device wait ran out (vertex %d, step %d)", st->h_abort[1],
                st->h_abort[2]);
  }
  out->stalled = code == 4;
  out->status = (code == 0) ? CONCORD_OK
                : (code == 1 || code == 4) ? CONCORD_NOT_CONVERGED
                : (code == 2) ? CONCORD_E_NONFINITE
                              : CONCORD_E_TIMEOUT;
  if (out->status == CONCORD_E_NONFINITE)
    return fail(CONCORD_E_NONFINITE, "non-finite objective or KKT residual after sweep %d",
                out->sweeps);
  return CONCORD_OK;
}

// Screened-sweep scratch, allocated on first use: Wb and V (p x ld of the
// FP64 width, so both precisions fit) and one block holding the candidate
// lists and per-candidate arrays, carved below.
struct ScreenLayout {
  size_t ctr, cand0, cand1, cnt_r0, cnt_r1, fail, off_r, cur_r, nd_pi, nd_pj, row_ent, term_ptr, term_pred, term_s, nd_rec, nd_delta, nd_new, nd_d2, jac,
      diag_old, omdiag_old, diag_new, dpart, dfill, diag_dd, pend_u, pend_d, pend_n, pend_new,
      rowacc, rowa_new, apart, loud, loudf, total;
};

ScreenLayout screen_layout(int p, int P, int nc, int tc) {
  ScreenLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ctr = take(sizeof(int) * kCtrs);
  L.cand0 = take(sizeof(int2) * (size_t)nc);
  L.cand1 = take(sizeof(int2) * (size_t)nc);
  L.cnt_r0 = take(sizeof(int) * (size_t)(p + 1));
  L.cnt_r1 = take(sizeof(int) * (size_t)(p + 1));
  L.fail = take(sizeof(int2) * (size_t)nc);
  L.off_r = take(sizeof(int) * (size_t)(p + 1));
  L.cur_r = take(sizeof(int) * (size_t)(p + 1));
  L.nd_pi = take(sizeof(int) * (size_t)nc);
  L.nd_pj = take(sizeof(int) * (size_t)nc);
  L.row_ent = take(sizeof(int) * 2 * (size_t)nc);
  L.term_ptr = take(sizeof(int) * ((size_t)nc + 1));
  L.term_pred = take(sizeof(int) * (size_t)tc);
  L.term_s = take(sizeof(double) * (size_t)tc);
  L.nd_rec = take(sizeof(double) * 4 * (size_t)nc);
  L.nd_delta = take(sizeof(double) * (size_t)nc);
  L.nd_new = take(sizeof(double) * (size_t)nc);
  L.nd_d2 = take(sizeof(double) * (size_t)nc);
  L.jac = take(sizeof(unsigned long long) * kJacMax);
  L.diag_old = take(sizeof(double) * (size_t)p);

  L.omdiag_old = take(sizeof(double) * (size_t)p);
  L.diag_new = take(sizeof(double) * (size_t)p);
  L.dpart = take(sizeof(double) * 1024);
  L.dfill = take(sizeof(int) * 1024);
  L.diag_dd = take(sizeof(double) * (size_t)p);
  L.pend_u = take(sizeof(int) * (size_t)p * kPendRow);
  L.pend_d = take(sizeof(double) * (size_t)p * kPendRow);
  L.pend_n = take(sizeof(int) * (size_t)p);
  L.pend_new = take(sizeof(int) * (size_t)p);
  L.rowacc = take(sizeof(double) * (size_t)p);
  L.rowa_new = take(sizeof(double) * (size_t)p);
  L.apart = take(sizeof(double) * 1024);
  L.loud = take(sizeof(int) * kLoudMax);
  L.loudf = take(sizeof(int) * (size_t)p);
  L.total = off;
  return L;
}

int ensure_screen(concord_state* st) {
  if (st->scr) return CONCORD_OK;
  const int p = st->p;
  const long long pairs = (long long)p * (p - 1) / 2;
  // every pair when there are at most 256k of them, else 16 per row
  // (states with a CTA budget, the concurrent stability workers: 64k)
  const bool budgeted = st->max_ctas > 0 && st->max_ctas < st->sms;
  long long nc = 16LL * p;
  if (nc < (budgeted ? 65536 : (1 << 18))) nc = budgeted ? 65536 : (1 << 18);
  if (nc > pairs) nc = pairs > 0 ? pairs : 1;
  st->nc_cap = (int)nc;
  // a row with k candidates carries k (k - 1) / 2 correction terms (12 bytes
  // each); a fixed-point round reads every term, so the list grows with p
  // (where a dense sweep's cost grows too) up to 32 M terms; a sweep whose
  // count exceeds it is handed to the dense kernel before any term is built.
  // A budgeted state (a fraction of the SMs) keeps 4 M: with few SMs the
  // longer screened sweeps lost to the dense kernel (measured on the
  // stability workload)
  long long tc = budgeted ? (1LL << 22) : 16384LL * p;
  if (tc > (1LL << 25)) tc = 1LL << 25;
  if (tc < 8 * nc) tc = 8 * nc;
  st->term_cap = (int)tc;
  const ScreenLayout L = screen_layout(p, st->P, st->nc_cap, st->term_cap);
  const size_t mat = (size_t)p * st->ld * sizeof(double);
  CK(cudaMalloc(&st->Wb, mat));
  CK(cudaMalloc(&st->V, mat));
  CK(cudaMalloc(&st->scr, L.total));
  CK(cudaMemsetAsync(st->Wb, 0, mat, st->stream));
  CK(cudaMemsetAsync(st->V, 0, mat, st->stream));
  int occ = 0;
  CK(screened_occupancy(is_mixed(st), &occ));
  if (occ < 1) return fail(CONCORD_E_OCCUPANCY, "screened sweep kernel cannot be resident");
  st->screened_grid = st->sms;  // one CTA per SM
  return CONCORD_OK;
}

template <typename T>
ScreenWork<T> screen_work(concord_state* st) {
  const ScreenLayout L = screen_layout(st->p, st->P, st->nc_cap, st->term_cap);
  char* b = (char*)st->scr;
  ScreenWork<T> w;
  w.ctr = (int*)(b + L.ctr);
  w.cand[0] = (int2*)(b + L.cand0);
  w.cand[1] = (int2*)(b + L.cand1);
  w.cnt_r[0] = (int*)(b + L.cnt_r0);
  w.cnt_r[1] = (int*)(b + L.cnt_r1);
  w.fail = (int2*)(b + L.fail);
  w.off_r = (int*)(b + L.off_r);
  w.cur_r = (int*)(b + L.cur_r);
  w.nd_pi = (int*)(b + L.nd_pi);
  w.nd_pj = (int*)(b + L.nd_pj);
  w.row_ent = (int*)(b + L.row_ent);
  w.term_ptr = (int*)(b + L.term_ptr);
  w.term_pred = (int*)(b + L.term_pred);
  w.term_s = (T*)(b + L.term_s);
  w.nd_rec = (T*)(b + L.nd_rec);
  w.nd_delta = (T*)(b + L.nd_delta);
  w.nd_new = (T*)(b + L.nd_new);
  w.nd_d2 = (T*)(b + L.nd_d2);
  w.jac = (unsigned long long*)(b + L.jac);
  w.diag_old = (T*)(b + L.diag_old);

  w.omdiag_old = (double*)(b + L.omdiag_old);
  w.diag_new = (double*)(b + L.diag_new);
  w.dpart = (double*)(b + L.dpart);
  w.dfill = (int*)(b + L.dfill);
  w.diag_dd = (T*)(b + L.diag_dd);
  w.pend_u = (int*)(b + L.pend_u);
  w.pend_d = (T*)(b + L.pend_d);
  w.pend_n = (int*)(b + L.pend_n);
  w.pend_new = (int*)(b + L.pend_new);
  w.rowacc = (double*)(b + L.rowacc);
  w.rowa_new = (double*)(b + L.rowa_new);
  w.apart = (double*)(b + L.apart);
  w.loud = (int*)(b + L.loud);
  w.loudf = (int*)(b + L.loudf);
  w.nc_cap = st->nc_cap;
  w.term_cap = st->term_cap;
  w.fail_cap = st->nc_cap;
  return w;
}

// Optional lambda path of a screened launch (device arrays).
struct PathArgs {
  const double* lam;
  int n, start;
  double* res;
  void* om;
  int ldo;
  float* cnt;
  int break_stall;  // a stalled lambda ends the launch (the host polishes it)
};

// One persistent launch of the screened sweep kernel; out->status_code is
// the kernel's status (kStatusDense: hand the next sweep to the dense kernel).
template <typename T>
int launch_screened_run(concord_state* st, T* S, T* W, T* Om, const T* sdiagT, double* omdiag64,
                        double lambda, double tol, int stop_rule, int n_sweeps, int kkt_only,
                        int hist_offset, int stall_stop, RunOut* out, int* code,
                        const PathArgs* path = nullptr) {
  int rc = ensure_screen(st);
  if (rc != CONCORD_OK) return rc;
  const ScreenLayout L = screen_layout(st->p, st->P, st->nc_cap, st->term_cap);
  // a list left by the previous launch (one-shot), else screen from scratch
  const int start_list = (!kkt_only && n_sweeps > 0 && !path) ? st->start_list : -1;
  const int start_scan = start_list >= 0 && st->start_scan ? 1 : 0;
  st->start_list = -1;
  st->start_scan = false;
  CK(cudaMemsetAsync(st->barrier, 0, sizeof(unsigned), st->stream));
  CK(cudaMemsetAsync(st->abort_info, 0, 3 * sizeof(int), st->stream));
  CK(cudaMemsetAsync((char*)st->scr + L.pend_n, 0, sizeof(int) * (size_t)st->p, st->stream));
  if (start_list < 0) {
    CK(cudaMemsetAsync((char*)st->scr + L.ctr, 0, sizeof(int) * kCtrs, st->stream));
    CK(cudaMemsetAsync((char*)st->scr + L.cnt_r0, 0, sizeof(int) * (size_t)(st->p + 1), st->stream));
    CK(cudaMemsetAsync((char*)st->scr + L.cnt_r1, 0, sizeof(int) * (size_t)(st->p + 1), st->stream));
  }
  ScreenArgs<T> a;
  memset(&a, 0, sizeof a);
  a.p = st->p;
  a.P = st->P;
  a.ld = st->ld;
  a.W = W;
  a.Wb = (T*)st->Wb;
  a.V = (T*)st->V;
  a.Om = Om;
  a.S = S;
  a.sdiag = sdiagT;
  a.sdiag64 = st->sdiag64;
  a.omdiag64 = omdiag64;
  a.w = screen_work<T>(st);
  a.barrier = st->barrier;
  a.wait.abort = st->abort_info;
  a.wait.info = st->abort_info + 1;
  a.wait.timeout_ns = (uint64_t)(st->timeout_s * 1e9);
  a.partials = st->partials;
  a.hist = st->hist + (size_t)hist_offset * kHist;
  a.hist_len = kHistCap - hist_offset;
  a.result = st->result;
  a.lambda = lambda;
  a.tol = tol;
  a.delta_tol = 1e-5;
  a.stop_rule = stop_rule;
  a.n_sweeps = n_sweeps;
  a.kkt_only = kkt_only;
  a.stall_stop = stall_stop;
  a.max_redo = 8;
  a.start_list = start_list;
  a.start_scan = start_scan;
  const bool check_flag = st->flag_pending;
  st->flag_pending = false;
  a.input_flag = check_flag ? st->flag : nullptr;
  a.mrow = st->mrow;
  a.lazy_verify = st->lazy_verify ? 1 : 0;
  a.keep_w = st->screen_keep_w ? 1 : 0;
  st->screen_keep_w = true;  // one-shot
  if (path) {
    a.path_lambda = path->lam;
    a.path_n = path->n;
    a.path_start = path->start;
    a.path_res = path->res;
    a.path_om = (T*)path->om;
    a.path_ldo = path->ldo;
    a.path_cnt = path->cnt;
    a.path_break_stall = path->break_stall;
  }
  st->last_variant = CONCORD_SWEEP_SCREENED;

  const int slot_ev = st->n_launch < kMaxTimedLaunches ? st->n_launch : -1;
  if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev], st->stream));
  CK(launch_screened(a, st->max_ctas > 0 && st->max_ctas < st->screened_grid ? st->max_ctas
                                                                              : st->screened_grid,
                     st->stream));
  if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev + 1], st->stream));
  CK(cudaMemcpyAsync(st->h_result, st->result, kRes * sizeof(double), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaMemcpyAsync(st->h_abort, st->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                     st->stream));
  if (check_flag)
    CK(cudaMemcpyAsync(st->h_flag, st->flag, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  if (check_flag && *st->h_flag != 0) {
    const int rc_in = input_flag_error(*st->h_flag);
    if (rc_in != CONCORD_OK) return rc_in;
  }
  const double* r = st->h_result;
  out->sweeps = (int)r[kResSweeps];
  out->kkt = r[kResKkt];
  out->obj = r[kResObj];
  out->delta = r[kResDelta];
  out->active = r[kResActive];
  out->first_delta = (int)r[kResFirstDelta];
  out->redos = (int)r[kResRedo];
  out->next_list = (int)r[kResList];
  out->lazy = (int)r[kResLazy];
  out->acc = r[kResAcc];
  out->partial = (int)r[kResPartial];
  if (slot_ev >= 0) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, st->lev[2 * slot_ev], st->lev[2 * slot_ev + 1]));
    st->launch_ms[slot_ev] = ms;
    st->launch_sweeps[slot_ev] = out->sweeps;
    st->n_launch = slot_ev + 1;
  }
  *code = (int)r[kResStatus];
  if (st->h_abort[0] != 0) {
    out->status = CONCORD_E_TIMEOUT;
    out->to_vertex = st->h_abort[1];
    out->to_step = st->h_abort[2];
    return fail(CONCORD_E_TIMEOUT, "device wait ran out (phase %d)", st->h_abort[2]);
  }
  out->stalled = *code == 4;
  out->status = (*code == 0) ? CONCORD_OK
                : (*code == 1 || *code == 4 || *code == kStatusDense) ? CONCORD_NOT_CONVERGED
                : (*code == 2) ? CONCORD_E_NONFINITE
                               : CONCORD_E_TIMEOUT;
  if (out->status == CONCORD_E_NONFINITE)
    return fail(CONCORD_E_NONFINITE, "non-finite objective or KKT residual after sweep %d",
                out->sweeps);
  return CONCORD_OK;
}

// Sweeps in the state's chosen variant.  Screened launches run until the
// stopping rule, the sweep budget, or a sweep whose candidates overflow the
// lists; such a sweep (and any following sweep that still changes more than
// half the list capacity) runs on the dense kernel, then screening resumes.
template <typename T>
int launch_run(concord_state* st, T* S, T* W, T* Om, const T* sdiagT, double* omdiag64, double lambda,
               double tol, int stop_rule, int n_sweeps, int kkt_only, int hist_offset, int stall_stop,
               RunOut* out) {
  const bool mixed = sizeof(T) == 4;
  const bool own = mixed == is_mixed(st);
  const int sv = st->sweep_variant;
  const bool screened = st->fault_vertex < 0 &&
                        (!own || sv == CONCORD_SWEEP_AUTO || sv == CONCORD_SWEEP_SCREENED);
  if (!screened)
    return launch_dense<T>(st, S, W, Om, sdiagT, omdiag64, lambda, tol, stop_rule, n_sweeps,
                           kkt_only, hist_offset, stall_stop, out);
  int done = 0, first_delta = 0, redos = 0, dense = 0;
  RunOut o;
  for (;;) {
    int code = 0;
    RunOut q;
    int rc = launch_screened_run<T>(st, S, W, Om, sdiagT, omdiag64, lambda, tol, stop_rule,
                                    n_sweeps - done, kkt_only, hist_offset + done, stall_stop, &q,
                                    &code);
    if (q.first_delta && !first_delta) first_delta = done + q.first_delta;
    done += q.sweeps;
    redos += q.redos;
    if (q.sweeps > 0 || kkt_only || code != kStatusDense) o = q;
    o.sweeps = done;
    o.first_delta = first_delta;
    o.redos = redos;
    o.dense_sweeps = dense;
    if (rc != CONCORD_OK || code != kStatusDense) {
      *out = o;
      if (rc == CONCORD_OK) out->status = q.status;
      return rc;
    }
    // dense sweeps until few enough pairs change
    for (;;) {
      if (done >= n_sweeps) {
        *out = o;
        out->status = CONCORD_NOT_CONVERGED;
        return CONCORD_OK;
      }
      RunOut dq;
      rc = launch_dense<T>(st, S, W, Om, sdiagT, omdiag64, lambda, tol, stop_rule, 1, 0,
                           hist_offset + done, 0, &dq, true);
      if (dq.first_delta && !first_delta) first_delta = done + dq.first_delta;
      done += dq.sweeps;
      dense += dq.sweeps;
      o = dq;
      o.sweeps = done;
      o.first_delta = first_delta;
      o.redos = redos;
      o.dense_sweeps = dense;
      if (rc != CONCORD_OK || dq.status != CONCORD_NOT_CONVERGED || dq.stalled ||
          done >= n_sweeps) {
        *out = o;
        return rc;
      }
      if (dq.active < 0.5 * st->nc_cap) break;
    }
  }
}

void fill_result(concord_result* res, const RunOut& o, int sweeps, int sweeps32, int first_delta,
                 double lambda, double seconds) {
  if (!res) return;
  memset(res, 0, sizeof *res);
  res->status = o.status;
  res->sweeps = sweeps;
  res->sweeps_fp32 = sweeps32;
  res->first_delta_sweep = first_delta;
  res->objective = o.obj;
  res->kkt = o.kkt;
  res->delta = o.delta;
  res->lambda = lambda;
  res->active_pairs = (long long)(o.active + 0.5);
  res->seconds = seconds;
  res->timeout_vertex = o.to_vertex;
  res->timeout_step = o.to_step;
  res->screen_redos = o.redos;
  res->dense_sweeps = o.dense_sweeps;
  res->s_refined = o.s_refined;
  res->lazy_sweeps = o.lazy;
  res->sparse_sweeps = o.sparse;
  res->partial_sweeps = o.partial;
}

int ensure_path(concord_state* st, int n_lambda, size_t n_rows) {
  if (n_lambda > st->path_cap) {
    if (st->path_lam) cudaFree(st->path_lam);
    if (st->path_res) cudaFree(st->path_res);
    st->path_lam = nullptr;
    st->path_res = nullptr;
    st->path_cap = 0;
    CK(cudaMalloc(&st->path_lam, sizeof(double) * n_lambda));
    CK(cudaMalloc(&st->path_res, sizeof(double) * kRes * n_lambda));
    st->path_cap = n_lambda;
  }
  if (n_rows > st->rows_cap) {
    if (st->rows_dev) cudaFree(st->rows_dev);
    st->rows_dev = nullptr;
    st->rows_cap = 0;
    CK(cudaMalloc(&st->rows_dev, sizeof(int) * n_rows));
    st->rows_cap = n_rows;
  }
  return CONCORD_OK;
}

void result_from_row(concord_result* r, const double* row, double lambda) {
  memset(r, 0, sizeof *r);
  const int code = (int)row[kResStatus];
  r->status = code == 0 ? CONCORD_OK : (code == 2 ? CONCORD_E_NONFINITE : CONCORD_NOT_CONVERGED);
  r->sweeps = (int)row[kResSweeps];
  r->first_delta_sweep = (int)row[kResFirstDelta];
  r->objective = row[kResObj];
  r->kkt = row[kResKkt];
  r->delta = row[kResDelta];
  r->lambda = lambda;
  r->active_pairs = (long long)(row[kResActive] + 0.5);
  r->timeout_vertex = r->timeout_step = -1;
  r->screen_redos = (int)row[kResRedo];
}

// The lambda path in the state's working precision (lambdas already in
// st->path_lam): one screened launch walks the lambdas, warm-starting each
// from the previous; a lambda whose sweeps need the dense kernel runs through
// the single-lambda dispatcher and the path resumes after it.
int demote_from_fp64(concord_state* st);

// A path lambda whose FP32 sweeps ended on the stall rule (the FP32 rounding
// floor, or progress too slow to tell apart from it): FP64 copies from the
// FP32 iterate (W rebuilt in FP64 from Omega and S64), FP64 sweeps to tol
// (at most `left`), then the FP32 working set back from the FP64 copies.
int polish_path_lambda(concord_state* st, double lambda, double tol, int left, RunOut* o2) {
  CK(launch_convert(st->Om, 1, st->ld, st->Om64, 0, st->ld, st->p, st->p, st->stream));
  CK(cudaMemcpy2DAsync(st->Om64, (size_t)(st->ld + 1) * sizeof(double), st->omdiag64,
                       sizeof(double), sizeof(double), st->p, cudaMemcpyDeviceToDevice,
                       st->stream));
  CK(launch_refresh_w(st->Om64, st->S64, st->W64, st->p, st->ld, st->sms, st->stream));
  st->w64_stale = false;
  const int start_list = st->start_list;
  st->start_list = -1;
  int rc = launch_run<double>(st, st->S64, st->W64, st->Om64, st->sdiag64, nullptr, lambda, tol,
                              CONCORD_STOP_KKT, left > 0 ? left : 1, 0, 0, 0, o2);
  st->start_list = start_list;
  if (rc != CONCORD_OK) return rc;
  return demote_from_fp64(st);
}

// Warm-started lambda path.  The screened kernel walks the lambdas in one
// launch until a lambda's candidates overflow (that lambda then runs on the
// single-lambda dispatcher and the path resumes after it) or, in mixed
// precision, until a lambda's FP32 sweeps stall (that lambda is polished in
// FP64 and the path resumes after it).
template <typename T>
int path_impl(concord_state* st, const double* lambdas, int n, double tol, int max_sweeps,
              concord_result* results, void* om_out, int ldo, float* cnt) {
  const bool mixed = sizeof(T) == 4;
  T* S = (T*)st->S;
  T* W = (T*)st->W;
  T* Om = (T*)st->Om;
  const T* sd = (const T*)st->sdiagT;
  double* omd = mixed ? st->omdiag64 : nullptr;
  std::vector<double> rows((size_t)kRes * n);
  int start = 0;
  st->n_launch = 0;
  // the lambda `k` is finished on the current iterate: its Omega and support
  auto finish = [&](int k, bool polished) -> int {
    if (om_out)
      CK(cudaMemcpy2DAsync((T*)om_out + (size_t)k * st->p * ldo, sizeof(T) * ldo, Om,
                           sizeof(T) * st->ld, sizeof(T) * st->p, st->p, cudaMemcpyDeviceToDevice,
                           st->stream));
    if (cnt) {
      if (polished)
        CK(launch_support_add(st->Om64, 0, st->ld, st->p, cnt + (size_t)k * st->p * st->p,
                              st->stream));
      else
        CK(launch_support_add(Om, mixed ? 1 : 0, st->ld, st->p, cnt + (size_t)k * st->p * st->p,
                              st->stream));
    }
    return CONCORD_OK;
  };
  const int brk = mixed && st->path_polish ? 1 : 0;
  while (start < n) {
    RunOut o;
    int code = 0;
    PathArgs pa{st->path_lam, n, start, st->path_res, om_out, ldo, cnt, brk};
    int rc = launch_screened_run<T>(st, S, W, Om, sd, omd, lambdas[start], tol, CONCORD_STOP_KKT,
                                    max_sweeps, 0, 0, mixed ? 1 : 0, &o, &code, &pa);
    if (rc != CONCORD_OK && rc != CONCORD_NOT_CONVERGED) return rc;
    CK(cudaMemcpy(rows.data(), st->path_res, sizeof(double) * kRes * n, cudaMemcpyDeviceToHost));
    const bool stalled = brk && code == 4;
    const int stop = (code == kStatusDense || stalled) ? (int)st->h_result[kResPath] : n;
    for (int k = start; k < stop && k < n; ++k)
      if (results) result_from_row(results + k, rows.data() + (size_t)kRes * k, lambdas[k]);
    if (code != kStatusDense && !stalled) break;
    // lambda `stop` on the dense-capable dispatcher (after the sweeps the
    // path launch already did at it), then the rest of the path
    int done = (int)st->h_result[kResSweeps];
    RunOut od = o;
    bool stall_now = stalled;
    if (code == kStatusDense) {
      rc = launch_run<T>(st, S, W, Om, sd, omd, lambdas[stop], tol, CONCORD_STOP_KKT,
                         max_sweeps > done ? max_sweeps - done : 1, 0, 0, mixed ? 1 : 0, &od);
      if (rc != CONCORD_OK) return rc;
      done += od.sweeps;
      stall_now = brk && od.stalled;
    }
    if (stall_now) {
      RunOut o2;
      if ((rc = polish_path_lambda(st, lambdas[stop], tol, max_sweeps - done, &o2)) != CONCORD_OK)
        return rc;
      if (results) fill_result(results + stop, o2, done + o2.sweeps, done, od.first_delta,
                               lambdas[stop], 0.0);
    } else if (results) {
      fill_result(results + stop, od, done, mixed ? done : 0, od.first_delta, lambdas[stop], 0.0);
    }
    if ((rc = finish(stop, stall_now)) != CONCORD_OK) return rc;
    start = stop + 1;
  }
  CK(cudaStreamSynchronize(st->stream));
  return CONCORD_OK;
}

// Buffers of the S refinement, sized for candidate lists of up to `list`
// pairs (allocated on first use, grown when needed).
int ensure_refine(concord_state* st, int list) {
  const int p = st->p;
  if (!st->rf.cnt) {
    CK(cudaMalloc(&st->rf.cnt, sizeof(int) * (size_t)(p + 1)));
    CK(cudaMalloc(&st->rf.off, sizeof(int) * (size_t)(p + 1)));
    CK(cudaMalloc(&st->rf.cur, sizeof(int) * (size_t)(p + 1)));
    CK(cudaMalloc(&st->rf.ctr, sizeof(int) * kRefineCtrs));
    CK(cudaMalloc(&st->rf.bitmap, sizeof(unsigned) * refine_bitmap_words(p)));
  }
  if (!st->rf.cand) {
    st->rf.cand_cap = 16 * p > (1 << 18) ? 16 * p : (1 << 18);
    CK(cudaMalloc(&st->rf.cand, sizeof(int2) * (size_t)st->rf.cand_cap));
  }
  const int need = 2 * (list > st->rf.cand_cap ? list : st->rf.cand_cap);
  if (need > st->rf.nbr_cap) {
    if (st->rf.nbr) cudaFree(st->rf.nbr);
    st->rf.nbr = nullptr;
    CK(cudaMalloc(&st->rf.nbr, sizeof(int) * (size_t)need));
    st->rf.nbr_cap = need;
  }
  return CONCORD_OK;
}

// mixed, S from data through a reduced-precision Gram: recompute the S
// entries that the stationarity conditions of the candidate pairs (list
// `list` of the screened kernel, or pairs collected from the FP32 iterate)
// read, in FP64 accuracy from the FP32 data (refine.cu), in both copies of
// S; then the diagonals and walk vectors derived from S.
int refine_s(concord_state* st, double lambda, int list) {
  const int p = st->p, ld = st->ld;
  const bool have_list = list >= 0 && st->scr != nullptr;
  int rc = ensure_refine(st, have_list ? st->nc_cap : 0);
  if (rc != CONCORD_OK) return rc;
  RefineArgs a;
  memset(&a, 0, sizeof a);
  a.p = p;
  a.ld = ld;
  a.n = st->zt_n;
  a.ldn = st->zt_ldn;
  a.sms = st->sms;
  a.zt = st->zt32;
  if (have_list) {
    const ScreenWork<float> w = screen_work<float>(st);
    a.cand = w.cand[list];
    a.n_cand = w.ctr + kCtrCand + list;
  }
  a.Om32 = (const float*)st->Om;
  a.W32 = (const float*)st->W;
  a.thr = (float)((1.0 - kRefineMargin) * lambda);
  a.own_cand = st->rf.cand;
  a.own_cap = st->rf.cand_cap;
  a.S64 = st->S64;
  a.S32 = (float*)st->S;
  a.nbr_cnt = st->rf.cnt;
  a.nbr_off = st->rf.off;
  a.nbr_cur = st->rf.cur;
  a.nbr = st->rf.nbr;
  a.bitmap = st->rf.bitmap;
  a.ctr = st->rf.ctr;
  a.mrow = st->mrow;
  CK(launch_refine_s(a, st->stream));
  CK(cudaMemcpyAsync(st->h_rf, st->rf.ctr + kRefineDone, sizeof(int), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(launch_extract_diag(st->S64, 0, ld, p, st->sdiag64, st->sdiagT, 1, st->flag, st->stream));
  CK(launch_subdiag(st->S64, 0, ld, p, st->P, st->sd1_64, st->sd2_64, st->stream));
  CK(launch_subdiag(st->S, 1, ld, p, st->P, st->sd1, st->sd2, st->stream));
  return CONCORD_OK;
}

// Buffers of the sparse polish for lists of up to st->nc_cap candidates and
// `term_cap` terms (one block, reallocated when the terms outgrow it).
int ensure_polish(concord_state* st, int term_cap) {
  if (st->pol.mem && st->pol.nc_cap >= st->nc_cap && st->pol.term_cap >= term_cap)
    return CONCORD_OK;
  if (st->pol.mem) cudaFree(st->pol.mem);
  st->pol.mem = nullptr;
  const size_t p = (size_t)st->p, nc = (size_t)st->nc_cap, tc = (size_t)term_cap;
  const size_t grid = (size_t)(st->max_grid > 0 ? st->max_grid : st->sms);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t ints = al(sizeof(int) * kPolCtrs) + al(8 * 3) + 3 * al(sizeof(int) * (p + 1)) +
                      al(sizeof(int) * p) + 3 * al(sizeof(int) * 2 * nc) + al(sizeof(int) * tc);
  const size_t dbls = al(8 * tc) + 5 * al(8 * nc) + al(8 * 2 * nc) + 4 * al(8 * p) + al(8 * grid) +
                      al(sizeof(int) * kPolLoudMax) + al(sizeof(int) * p);
  char* m = nullptr;
  CK(cudaMalloc((void**)&m, ints + dbls));
  st->pol.mem = m;
  st->pol.nc_cap = st->nc_cap;
  st->pol.term_cap = term_cap;
  PolishWork& w = st->pol.w;
  size_t o = 0;
  auto take = [&](size_t b) { char* r = m + o; o += al(b); return (void*)r; };
  w.ctr = (int*)take(sizeof(int) * kPolCtrs);
  w.rslot = (unsigned long long*)take(8 * 3);
  w.deg = (int*)take(sizeof(int) * (p + 1));
  w.off = (int*)take(sizeof(int) * (p + 1));
  w.toff = (int*)take(sizeof(int) * (p + 1));
  w.cur = (int*)take(sizeof(int) * p);
  w.ent0 = (int*)take(sizeof(int) * 2 * nc);
  w.ent = (int*)take(sizeof(int) * 2 * nc);
  w.pos = (int*)take(sizeof(int) * 2 * nc);
  w.term_q = (int*)take(sizeof(int) * tc);
  w.term_s = (double*)take(8 * tc);
  w.om = (double*)take(8 * nc);
  w.den = (double*)take(8 * nc);
  w.d0 = (double*)take(8 * nc);
  w.d1 = (double*)take(8 * nc);
  w.nw = (double*)take(8 * nc);
  w.base = (double*)take(8 * 2 * nc);
  w.diag = (double*)take(8 * p);
  w.diag_new = (double*)take(8 * p);
  w.dpart = (double*)take(8 * grid);
  w.rowa = (double*)take(8 * p);
  w.rowb = (double*)take(8 * p);
  w.loud = (int*)take(sizeof(int) * kPolLoudMax);
  w.loudf = (int*)take(sizeof(int) * p);
  w.nc_cap = st->nc_cap;
  w.term_cap = term_cap;
  return CONCORD_OK;
}

// The sparse FP64 polish (polish.cu) of the promoted iterate, on candidate
// list `list` of the FP32 launch with its accumulated bound `acc`.  *code is
// the kernel's status: 0 / 1 / 2 / 3 as the sweep kernels, kStatusNeedW when
// the bound (or the fixed point) failed before a sweep was committed (the
// sweeps already done stand; W must be rebuilt for the rest).
int polish_sparse(concord_state* st, double lambda, double tol, int stop_rule, int n_sweeps,
                  int hist_offset, int list, double acc, RunOut* out, int* code) {
  int term_cap = st->pol.term_cap > 0 ? st->pol.term_cap : 16 * st->nc_cap;
  const ScreenWork<float> sw = screen_work<float>(st);
  for (int attempt = 0;; ++attempt) {
    int rc = ensure_polish(st, term_cap);
    if (rc != CONCORD_OK) return rc;
    const PolishWork& w = st->pol.w;
    CK(cudaMemsetAsync(w.ctr, 0, sizeof(int) * kPolCtrs, st->stream));
    CK(cudaMemsetAsync(w.rslot, 0, 8 * 3, st->stream));
    CK(cudaMemsetAsync(w.deg, 0, sizeof(int) * (size_t)(st->p + 1), st->stream));
    CK(cudaMemsetAsync(st->barrier, 0, sizeof(unsigned), st->stream));
    CK(cudaMemsetAsync(st->abort_info, 0, 3 * sizeof(int), st->stream));
    PolishArgs a;
    memset(&a, 0, sizeof a);
    a.p = st->p;
    a.P = st->P;
    a.ld = st->ld;
    a.Om = st->Om64;
    a.Om32 = (const float*)st->Om;
    a.omdiag = st->omdiag64;
    a.S = st->S64;
    a.sdiag = st->sdiag64;
    a.mrow = st->mrow;
    a.cand = sw.cand[list];
    a.n_cand = sw.ctr + kCtrCand + list;
    a.ds_bits = (st->refine && st->zt_valid && st->rf.ctr) ? st->rf.ctr + kRefineDs : nullptr;
    a.acc0 = acc;
    a.rowacc = sw.rowacc;  // the FP32 launch's per-row bound on this list
    a.w = w;
    a.barrier = st->barrier;
    a.wait.abort = st->abort_info;
    a.wait.info = st->abort_info + 1;
    a.wait.timeout_ns = (uint64_t)(st->timeout_s * 1e9);
    a.partials = st->partials;
    a.hist = st->hist + (size_t)hist_offset * kHist;
    a.hist_len = kHistCap - hist_offset;
    a.result = st->result;
    a.lambda = lambda;
    a.tol = tol;
    a.delta_tol = 1e-5;
    a.stop_rule = stop_rule;
    a.n_sweeps = n_sweeps;
    const int slot_ev = st->n_launch < kMaxTimedLaunches ? st->n_launch : -1;
    if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev], st->stream));
    const int grid = st->max_ctas > 0 && st->max_ctas < st->sms ? st->max_ctas : st->sms;
    CK(launch_polish(a, grid, st->stream));
    if (slot_ev >= 0) CK(cudaEventRecord(st->lev[2 * slot_ev + 1], st->stream));
    CK(cudaMemcpyAsync(st->h_result, st->result, kRes * sizeof(double), cudaMemcpyDeviceToHost,
                       st->stream));
    CK(cudaMemcpyAsync(st->h_abort, st->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                       st->stream));
    CK(cudaMemcpyAsync(st->h_flag, w.ctr + kPolOverflow, sizeof(int), cudaMemcpyDeviceToHost,
                       st->stream));
    CK(cudaStreamSynchronize(st->stream));
    CK(cudaGetLastError());
    const double* r = st->h_result;
    *code = (int)r[kResStatus];
    if (*code == kStatusCapacity) {
      // the terms did not fit: grow once to what they need (bounded), else
      // leave the polish to the screened kernel
      const int need = *st->h_flag;
      if (attempt == 0 && need > term_cap && need <= (1 << 26)) {
        term_cap = need;
        continue;
      }
      *code = kStatusNeedW;
    }
    if (slot_ev >= 0) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, st->lev[2 * slot_ev], st->lev[2 * slot_ev + 1]));
      st->launch_ms[slot_ev] = ms;
      st->launch_sweeps[slot_ev] = (int)r[kResSweeps];
      st->n_launch = slot_ev + 1;
    }
    out->sweeps = (int)r[kResSweeps];
    out->kkt = r[kResKkt];
    out->obj = r[kResObj];
    out->delta = r[kResDelta];
    out->active = r[kResActive];
    out->first_delta = (int)r[kResFirstDelta];
    out->redos = 0;
    out->next_list = -1;
    out->lazy = (int)r[kResLazy];
    out->acc = r[kResAcc];
    out->partial = (int)r[kResPartial];
    if (st->h_abort[0] != 0) {
      out->status = CONCORD_E_TIMEOUT;
      out->to_vertex = st->h_abort[1];
      out->to_step = st->h_abort[2];
      return fail(CONCORD_E_TIMEOUT, "device wait ran out (phase %d)", st->h_abort[2]);
    }
    out->status = *code == 0 ? CONCORD_OK
                  : *code == 2 ? CONCORD_E_NONFINITE
                               : CONCORD_NOT_CONVERGED;
    if (*code == 2)
      return fail(CONCORD_E_NONFINITE, "non-finite objective or KKT residual after sweep %d",
                  out->sweeps);
    return CONCORD_OK;
  }
}

// mixed: W64 = Omega64 S64 again where a sparse polish left it out of date
int ensure_w64(concord_state* st) {
  if (!st->w64_stale) return CONCORD_OK;
  CK(launch_refresh_w(st->Om64, st->S64, st->W64, st->p, st->ld, st->sms, st->stream));
  st->w64_stale = false;
  return CONCORD_OK;
}

// mixed: FP32 iterate -> FP64 copies (Omega with its FP64 diagonal; W rebuilt
// in FP64 from Omega and S, after the S refinement when it applies)
int promote_to_fp64(concord_state* st, double lambda, int list, bool rebuild_w = true) {
  *st->h_rf = 0;
  if (st->refine && st->zt_valid) {
    int rc = refine_s(st, lambda, list);
    if (rc != CONCORD_OK) return rc;
  }
  if (rebuild_w) {
    CK(launch_convert(st->Om, 1, st->ld, st->Om64, 0, st->ld, st->p, st->p, st->stream));
    CK(cudaMemcpy2DAsync(st->Om64, (size_t)(st->ld + 1) * sizeof(double), st->omdiag64,
                         sizeof(double), sizeof(double), st->p, cudaMemcpyDeviceToDevice,
                         st->stream));
    CK(launch_refresh_w(st->Om64, st->S64, st->W64, st->p, st->ld, st->sms, st->stream));
  } else {
    // the sparse polish takes Omega from the FP32 iterate (its nonzeros are
    // candidates of the list) and writes the FP64 candidates and diagonal
    // into a zeroed FP64 Omega
    CK(cudaMemsetAsync(st->Om64, 0, sizeof(double) * (size_t)st->p * st->ld, st->stream));
  }
  st->w64_stale = !rebuild_w;
  st->om64_current = true;
  return CONCORD_OK;
}

// mixed: FP64 copies -> FP32 working set
int demote_from_fp64(concord_state* st) {
  int rc = ensure_w64(st);
  if (rc != CONCORD_OK) return rc;
  CK(launch_convert(st->Om64, 0, st->ld, st->Om, 1, st->ld, st->p, st->p, st->stream));
  CK(launch_convert(st->W64, 0, st->ld, st->W, 1, st->ld, st->p, st->p, st->stream));
  CK(cudaMemcpy2DAsync(st->omdiag64, sizeof(double), st->Om64, (size_t)(st->ld + 1) * sizeof(double),
                       sizeof(double), st->p, cudaMemcpyDeviceToDevice, st->stream));
  return CONCORD_OK;
}

int run_impl(concord_state* st, double lambda, double tol, int max_sweeps, int stop_rule,
             double switch_tol, int exact, concord_result* res) {
  if (!(lambda >= 0.0) || max_sweeps < 0 || (stop_rule != 0 && stop_rule != 1))
    return fail(CONCORD_E_ARG, "lambda >= 0, max_sweeps >= 0, stop_rule in {0,1} required");
  if (!exact && !(tol > 0.0)) return fail(CONCORD_E_ARG, "tol must be > 0");
  const double run_tol = exact ? -1.0 : tol;
  // a start screen of this state's current S and starting point (one-shot)
  const bool pre = st->prescreen && st->prescreen_lambda == lambda && is_mixed(st);
  st->prescreen = false;
  if (st->flag_pending && !pre) {  // the data checks, read here after all
    st->flag_pending = false;
    int bad = 0, rc0 = read_flag(st, &bad);
    if (rc0 != CONCORD_OK) return rc0;
    if ((rc0 = input_flag_error(bad)) != CONCORD_OK) return rc0;
  }
  st->hist_rows = 0;
  st->n_launch = 0;
  CK(cudaEventRecord(st->ev0, st->stream));
  RunOut o1, o2;
  int rc;
  if (!is_mixed(st)) {
    rc = launch_run<double>(st, st->S64, st->W64, st->Om64, (const double*)st->sdiagT, nullptr,
                            lambda, run_tol, stop_rule, max_sweeps, 0, 0, 0, &o1);
    CK(cudaEventRecord(st->ev1, st->stream));
    CK(cudaEventSynchronize(st->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
    st->hist_rows = o1.sweeps;
    fill_result(res, o1, o1.sweeps, 0, o1.first_delta, lambda, ms * 1e-3);
    return rc != CONCORD_OK ? rc : o1.status;
  }
  // mixed precision: FP32 sweeps until the rule holds at the switch
  // tolerance (default max(3 tol, 1e-5)) or the FP32 iteration stalls at
  // its rounding floor ...
  double tol1 = exact ? -1.0 : (switch_tol > 0 ? switch_tol : (3.0 * tol > 1e-5 ? 3.0 * tol : 1e-5));
  if (!exact && tol1 < tol) tol1 = tol;
  // the FP32 working set follows the FP64 copies lazily (after a polish)
  if (st->om64_current && (rc = demote_from_fp64(st)) != CONCORD_OK) return rc;
  // the one-pass start screened the starting point for this lambda: the
  // FP32 launch starts from that list (its first build scans the counts)
  const int sv0 = st->sweep_variant;
  if (pre && st->fault_vertex < 0 && (sv0 == CONCORD_SWEEP_AUTO || sv0 == CONCORD_SWEEP_SCREENED)) {
    st->start_list = 0;
    st->start_scan = true;
  }
  // the polish rebuilds W in FP64 from Omega: the FP32 launch need not bring
  // W up to date at its end (deferred updates of lazy sweeps may be dropped)
  st->screen_keep_w = exact != 0;
  rc = launch_run<float>(st, (float*)st->S, (float*)st->W, (float*)st->Om,
                         (const float*)st->sdiagT, st->omdiag64, lambda, tol1, stop_rule,
                         max_sweeps, 0, 0, exact ? 0 : 1, &o1);
  st->screen_keep_w = true;
  st->start_list = -1;  // one-shot, also when the sweeps did not take it
  st->start_scan = false;
  st->om64_current = false;
  st->hist_rows = o1.sweeps;
  if (rc != CONCORD_OK || exact) {
    CK(cudaEventRecord(st->ev1, st->stream));
    CK(cudaEventSynchronize(st->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
    fill_result(res, o1, o1.sweeps, o1.sweeps, o1.first_delta, lambda, ms * 1e-3);
    return rc != CONCORD_OK ? rc : o1.status;
  }
  // ... then FP64 polishing from W rebuilt in FP64, its first sweep on the
  // candidate list the FP32 phase left (same lambda)
  // (sparse polish: sweeps on the candidates alone while the lazy bound
  // holds, W not rebuilt; the screened polish from a rebuilt W otherwise, or
  // for the sweeps left when the bound fails)
  const int left = max_sweeps - o1.sweeps;
  const bool sparse = st->sparse_polish && left > 0 && o1.next_list >= 0;
  if ((rc = promote_to_fp64(st, lambda, o1.next_list, !sparse)) != CONCORD_OK) return rc;
  int code = kStatusNeedW, done = 0;
  if (sparse) {
    rc = polish_sparse(st, lambda, tol, stop_rule, left, o1.sweeps, o1.next_list, o1.acc, &o2,
                       &code);
    done = o2.sweeps;
    o2.sparse = done;
  }
  if (rc == CONCORD_OK && code == kStatusNeedW) {
    if ((rc = ensure_w64(st)) != CONCORD_OK) return rc;
    const int left2 = left - done;
    RunOut o3;
    st->start_list = left2 > 0 ? o1.next_list : -1;
    rc = launch_run<double>(st, st->S64, st->W64, st->Om64, st->sdiag64, nullptr, lambda, tol,
                            stop_rule, left2, left2 == 0 ? 1 : 0, o1.sweeps + done, 0, &o3);
    st->start_list = -1;
    if (done > 0) {
      o3.first_delta = o2.first_delta ? o2.first_delta : (o3.first_delta ? done + o3.first_delta : 0);
      o3.sweeps += done;
      o3.lazy += o2.lazy;
    }
    o3.sparse = done;
    o2 = o3;
  }
  st->hist_rows = o1.sweeps + o2.sweeps;
  // the FP64 copies now hold the iterate (om64_current); the FP32 working
  // set is refreshed from them when an FP32 phase next needs it
  CK(cudaEventRecord(st->ev1, st->stream));
  CK(cudaEventSynchronize(st->ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
  const int fd = o1.first_delta ? o1.first_delta : (o2.first_delta ? o1.sweeps + o2.first_delta : 0);
  o2.redos += o1.redos;
  o2.dense_sweeps += o1.dense_sweeps;
  o2.lazy += o1.lazy;
  o2.partial += o1.partial;
  o2.s_refined = *st->h_rf;  // read back by the polish launch's synchronisation
  fill_result(res, o2, o1.sweeps + o2.sweeps, o1.sweeps, fd, lambda, ms * 1e-3);
  return rc != CONCORD_OK ? rc : o2.status;
}

// Load S (already in the state's S64 for fp64, or S (f32) + S64 for mixed)
// bookkeeping: diagonals, Omega = I, W = S.
int reset_iterate(concord_state* st) {
  const int p = st->p, ld = st->ld;
  st->prescreen = false;
  CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  CK(launch_extract_diag(st->S64, 0, ld, p, st->sdiag64, is_mixed(st) ? st->sdiagT : nullptr, 1,
                         st->flag, st->stream));
  if (!is_mixed(st))
    CK(cudaMemcpyAsync(st->sdiagT, st->sdiag64, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                       st->stream));
  CK(launch_subdiag(st->S64, 0, ld, p, st->P, st->sd1_64, st->sd2_64, st->stream));
  if (is_mixed(st)) CK(launch_subdiag(st->S, 1, ld, p, st->P, st->sd1, st->sd2, st->stream));
  // row bounds of S for the screened kernel's lazy verification (from the
  // working-precision S; they bound the FP64 copy too)
  CK(launch_row_absmax(is_mixed(st) ? st->S : (const void*)st->S64, is_mixed(st) ? 1 : 0, ld, p,
                       st->mrow, st->stream));
  if (is_mixed(st)) {
    CK(launch_set_identity(st->Om, 1, p, ld, st->stream));
    CK(cudaMemcpyAsync(st->W, st->S, sizeof(float) * (size_t)p * ld, cudaMemcpyDeviceToDevice,
                       st->stream));
    CK(launch_fill_f64(st->omdiag64, 1.0, p, st->stream));
  } else {
    CK(launch_set_identity(st->Om64, 0, p, ld, st->stream));
    CK(cudaMemcpyAsync(st->W64, st->S64, sizeof(double) * (size_t)p * ld, cudaMemcpyDeviceToDevice,
                       st->stream));
  }
  st->om64_current = false;
  int bad = 0;
  int rc = read_flag(st, &bad);
  if (rc) return rc;
  if (bad & 2) return fail(CONCORD_E_NONFINITE, "S has a non-finite diagonal entry");
  if (bad & 1) return fail(CONCORD_E_NONPOS_DIAG, "S has a diagonal entry <= 0 (constant column?)");
  return CONCORD_OK;
}

}  // namespace

extern "C" {

size_t concord_result_size(void) { return sizeof(concord_result); }

const char* concord_last_error(void) { return g_err.c_str(); }

const char* concord_version(void) { return "concord-gb300 0.1 (sm_103a)"; }

int concord_schedule(int p, int32_t* pairs_host, int* n_colours) {
  if (p < 2 || !pairs_host || !n_colours) return fail(CONCORD_E_ARG, "p >= 2 and non-NULL outputs");
  const int pe = p + (p & 1), P = pe - 1, half = pe / 2;
  // slot q of colour c holds the vertices at facing ring positions; the
  // 0-based vertex at position m (1-based, m >= 2) during colour c is
  // ((m - 2 - c) mod P) + 1, and position 1 holds vertex 0
  for (int c = 0; c < P; ++c)
    for (int q = 0; q < half; ++q) {
      int u, v;
      if (q == 0) {
        u = 0;
        v = cm_partner(0, c, P);
      } else {
        // position m = q + 1 (1-based) faces position pe - q
        int m = q + 1;
        u = ((m - 2 - c) % P + P) % P + 1;
        v = cm_partner(u, c, P);
      }
      int32_t* slot = pairs_host + ((size_t)c * half + q) * 2;
      if (u >= p || v >= p) {
        slot[0] = slot[1] = -1;
      } else {
        slot[0] = u;
        slot[1] = v;
      }
    }
  *n_colours = P;
  return CONCORD_OK;
}

int concord_create(concord_state** out, int p, int precision, int n_cap, int device) {
  if (!out) return fail(CONCORD_E_ARG, "out is NULL");
  *out = nullptr;
  if (p < 2) return fail(CONCORD_E_ARG, "p must be >= 2 (got %d)", p);
  if (precision != CONCORD_FP64 && precision != CONCORD_MIXED)
    return fail(CONCORD_E_ARG, "precision must be CONCORD_FP64 or CONCORD_MIXED");
  if (n_cap < 0) return fail(CONCORD_E_ARG, "n_cap must be >= 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(CONCORD_E_CUDA, "no CUDA device");
  if (device < 0) CK(cudaGetDevice(&device));
  if (device >= ndev) return fail(CONCORD_E_ARG, "device %d out of range", device);
  CK(cudaSetDevice(device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(CONCORD_E_CUDA, "library is built for sm_103a; device is sm_%d%d", prop.major,
                prop.minor);
  if (!prop.cooperativeLaunch) return fail(CONCORD_E_CUDA, "device lacks cooperative launch");

  concord_state* st = new concord_state();
  st->device = device;
  st->sms = prop.multiProcessorCount;
  st->p = p;
  st->pe = p + (p & 1);
  st->P = st->pe - 1;
  st->ld = round_up(p, kTile);
  st->precision = precision;
  st->n_cap = n_cap;
  const size_t mat = (size_t)p * st->ld;
  const size_t e = is_mixed(st) ? 4 : 8;
  int rc = CONCORD_OK;
#define ALLOC(ptr, bytes)                                                       \
  do {                                                                          \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                       \
    if (e_ != cudaSuccess) {                                                    \
      rc = fail(CONCORD_E_NOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes),        \
                cudaGetErrorString(e_));                                        \
      goto fail_out;                                                            \
    }                                                                           \
  } while (0)
  {
    if (cudaStreamCreateWithFlags(&st->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(CONCORD_E_CUDA, "cudaStreamCreate failed");
      goto fail_out;
    }
    st->stream = st->own_stream;
    if (is_mixed(st)) {
      ALLOC(st->S, mat * e);
      ALLOC(st->W, mat * e);
      ALLOC(st->Om, mat * e);
      ALLOC(st->sdiagT, sizeof(float) * p);
      ALLOC(st->omdiag64, sizeof(double) * p);
      ALLOC(st->S64, mat * 8);
      ALLOC(st->W64, mat * 8);
      ALLOC(st->Om64, mat * 8);
    } else {
      ALLOC(st->S64, mat * 8);
      ALLOC(st->W64, mat * 8);
      ALLOC(st->Om64, mat * 8);
      ALLOC(st->sdiagT, sizeof(double) * p);
      st->S = st->S64;
      st->W = st->W64;
      st->Om = st->Om64;
    }
    ALLOC(st->sdiag64, sizeof(double) * p);
    ALLOC(st->mrow, sizeof(float) * p);
    ALLOC(st->sd1_64, sizeof(double) * p);
    ALLOC(st->sd2_64, sizeof(double) * p);
    if (is_mixed(st)) {
      ALLOC(st->sd1, sizeof(float) * p);
      ALLOC(st->sd2, sizeof(float) * p);
    }
    // mailboxes sized for the FP64 form (2 words) so both precisions fit
    ALLOC(st->mbox, sizeof(unsigned long long) * 2 * (size_t)st->depth * st->pe);
    cudaMemset(st->mbox, 0, sizeof(unsigned long long) * 2 * (size_t)st->depth * st->pe);
    ALLOC(st->barrier, sizeof(unsigned));
    ALLOC(st->abort_info, 3 * sizeof(int));
    ALLOC(st->flag, sizeof(int));
    ALLOC(st->lmax, sizeof(unsigned long long));
    st->max_grid = st->sms * 32;
    ALLOC(st->partials, sizeof(double) * kParts * (size_t)st->max_grid);
    ALLOC(st->hist, sizeof(double) * kHist * (size_t)kHistCap);
    ALLOC(st->result, sizeof(double) * kRes);
    ALLOC(st->mean, sizeof(double) * p);
    ALLOC(st->inv_scale, sizeof(double) * p);
    if (n_cap > 0) {
      st->ldz = st->ld;
      ALLOC(st->Z, (size_t)n_cap * st->ldz * e);
      ALLOC(st->Xstage, (size_t)n_cap * p * sizeof(double));
      st->n_pad = round_up(n_cap, 64);
      st->p_pad = round_up(p, 128);
      if (is_mixed(st)) {
        ALLOC(st->zt_hi, sizeof(float) * (size_t)st->n_pad * st->p_pad);
        ALLOC(st->zt_lo, sizeof(float) * (size_t)st->n_pad * st->p_pad);
        ALLOC(st->zt32, sizeof(float) * (size_t)round_up(n_cap, 32) * st->p_pad);
      }
    }
    st->gram_mode = is_mixed(st) ? CONCORD_GRAM_TF32X3 : CONCORD_GRAM_FP64;
    if (cudaMallocHost((void**)&st->h_result, sizeof(double) * kRes) != cudaSuccess ||
        cudaMallocHost((void**)&st->h_abort, 3 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&st->h_flag, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&st->h_rf, sizeof(int)) != cudaSuccess) {
      rc = fail(CONCORD_E_NOMEM, "cudaMallocHost failed");
      goto fail_out;
    }
    if (cudaEventCreate(&st->ev0) != cudaSuccess || cudaEventCreate(&st->ev1) != cudaSuccess) {
      rc = fail(CONCORD_E_CUDA, "cudaEventCreate failed");
      goto fail_out;
    }
    for (int q = 0; q < 2 * kMaxTimedLaunches; ++q)
      if (cudaEventCreate(&st->lev[q]) != cudaSuccess) {
        rc = fail(CONCORD_E_CUDA, "cudaEventCreate failed");
        goto fail_out;
      }
    if (cudaDeviceSynchronize() != cudaSuccess) {
      rc = fail(CONCORD_E_CUDA, "device sync after allocation failed");
      goto fail_out;
    }
    // Omega = I, W = S = I until concord_set_S
    if (is_mixed(st)) {
      launch_set_identity(st->S, 1, p, st->ld, st->stream);
      launch_set_identity(st->S64, 0, p, st->ld, st->stream);
    } else {
      launch_set_identity(st->S64, 0, p, st->ld, st->stream);
    }
    rc = reset_iterate(st);
    if (rc != CONCORD_OK) goto fail_out;
    *out = st;
    return CONCORD_OK;
  }
#undef ALLOC
fail_out:
  concord_destroy(st);
  return rc;
}

int concord_destroy(concord_state* st) {
  if (!st) return CONCORD_OK;
  cudaSetDevice(st->device);
  if (st->stream) cudaStreamSynchronize(st->stream);
  void* dev[] = {st->path_lam, st->path_res, st->rows_dev, st->Wb, st->V, st->scr, st->sd1_64, st->sd2_64, st->mbox, st->barrier, st->abort_info, st->flag, st->lmax, st->partials,
                 st->hist, st->result, st->mean, st->inv_scale, st->Z, st->Xstage, st->zt_hi,
                 st->zt_lo, st->sdiag64, st->sdiagT, st->omdiag64, st->S64, st->W64, st->Om64,
                 st->zt32, st->rf.cnt, st->rf.off, st->rf.cur, st->rf.nbr, st->rf.ctr, st->rf.cand,
                 st->rf.bitmap, st->mrow, st->pol.mem};
  for (void* d : dev)
    if (d) cudaFree(d);
  void* adj_dev[] = {st->adj.cnt, st->adj.rowptr, st->adj.bad, st->adj.col, st->adj.erow,
                     st->adj.mirror, st->adj.om, st->adj.minv, st->adj.b, st->adj.x, st->adj.r,
                     st->adj.z, st->adj.p0, st->adj.p1, st->adj.q, st->adj.scal, st->adj.Z,
                     st->adj.P, st->adj.Q, st->adj.dZ, st->adj.part1, st->adj.part2, st->adj.m1,
                     st->adj.m2, st->adj.mean, st->adj.scale};
  for (void* d : adj_dev)
    if (d) cudaFree(d);
  void* csr_dev[] = {st->csr_cnt, st->csr_rowptr, st->csr_col, st->csr_row, st->csr_val};
  for (void* d : csr_dev)
    if (d) cudaFree(d);
  if (is_mixed(st)) {
    if (st->sd1) cudaFree(st->sd1);
    if (st->sd2) cudaFree(st->sd2);
    if (st->S) cudaFree(st->S);
    if (st->W) cudaFree(st->W);
    if (st->Om) cudaFree(st->Om);
  }
  if (st->h_result) cudaFreeHost(st->h_result);
  if (st->h_abort) cudaFreeHost(st->h_abort);
  if (st->h_flag) cudaFreeHost(st->h_flag);
  if (st->h_rf) cudaFreeHost(st->h_rf);
  if (st->ev0) cudaEventDestroy(st->ev0);
  if (st->ev1) cudaEventDestroy(st->ev1);
  for (int q = 0; q < 2 * kMaxTimedLaunches; ++q)
    if (st->lev[q]) cudaEventDestroy(st->lev[q]);
  if (st->own_stream) cudaStreamDestroy(st->own_stream);
  delete st;
  return CONCORD_OK;
}

int concord_set_stream(concord_state* st, void* stream) {
  int rc = check_state(st);
  if (rc) return rc;
  st->stream = stream ? (cudaStream_t)stream : st->own_stream;
  return CONCORD_OK;
}

int concord_set_timeout(concord_state* st, double seconds) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (!(seconds > 0.0) || seconds > 3600.0) return fail(CONCORD_E_ARG, "timeout must be in (0, 3600] s");
  st->timeout_s = seconds;
  return CONCORD_OK;
}

int concord_set_fault(concord_state* st, int vertex, int step) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (vertex >= st->p) return fail(CONCORD_E_ARG, "vertex out of range");
  st->fault_vertex = vertex < 0 ? -1 : vertex;
  st->fault_step = vertex < 0 ? -1 : step;
  return CONCORD_OK;
}

int concord_set_S(concord_state* st, const void* S_dev, int s_dtype, int lds) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!S_dev || (s_dtype != CONCORD_F64 && s_dtype != CONCORD_F32) || lds < st->p)
    return fail(CONCORD_E_ARG, "S_dev non-NULL, dtype F64/F32, lds >= p required");
  const int p = st->p, ld = st->ld, f32 = s_dtype == CONCORD_F32;
  CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  CK(launch_check_symmetric(S_dev, f32, p, lds, st->flag, st->stream));
  int bad = 0;
  if ((rc = read_flag(st, &bad))) return rc;
  if (bad & 2) return fail(CONCORD_E_NONFINITE, "S has a non-finite entry");
  if (bad & 1) return fail(CONCORD_E_ARG, "S is not symmetric");
  st->zt_valid = false;  // no data behind this S: nothing to refine from
  CK(launch_convert(S_dev, f32, lds, st->S64, 0, ld, p, p, st->stream));
  if (is_mixed(st)) CK(launch_convert(S_dev, f32, lds, st->S, 1, ld, p, p, st->stream));
  return reset_iterate(st);
}

int concord_set_omega(concord_state* st, const void* Om_dev, int dtype, int ld_in) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!Om_dev || (dtype != CONCORD_F64 && dtype != CONCORD_F32) || ld_in < st->p)
    return fail(CONCORD_E_ARG, "Omega0 non-NULL, dtype F64/F32, ld >= p required");
  const int p = st->p, ld = st->ld, f32 = dtype == CONCORD_F32;
  st->prescreen = false;
  CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  CK(launch_check_symmetric(Om_dev, f32, p, ld_in, st->flag, st->stream));
  CK(launch_extract_diag(Om_dev, f32, ld_in, p, nullptr, nullptr, 0, st->flag, st->stream));
  int bad = 0;
  if ((rc = read_flag(st, &bad))) return rc;
  if (bad & 2) return fail(CONCORD_E_NONFINITE, "Omega0 has a non-finite entry");
  if (bad & 1) return fail(CONCORD_E_ARG, "Omega0 is not symmetric with a positive diagonal");
  CK(launch_convert(Om_dev, f32, ld_in, st->Om64, 0, ld, p, p, st->stream));
  CK(launch_refresh_w(st->Om64, st->S64, st->W64, p, ld, st->sms, st->stream));
  st->w64_stale = false;
  if (is_mixed(st)) {
    st->om64_current = true;
    if ((rc = demote_from_fp64(st))) return rc;
  }
  CK(cudaStreamSynchronize(st->stream));
  return CONCORD_OK;
}

static int get_matrix(concord_state* st, bool omega, void* out, int dtype, int ld_out) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!out || (dtype != CONCORD_F64 && dtype != CONCORD_F32) || ld_out < st->p)
    return fail(CONCORD_E_ARG, "out non-NULL, dtype F64/F32, ld >= p required");
  const int p = st->p, ld = st->ld, f32 = dtype == CONCORD_F32;
  if (!is_mixed(st) || st->om64_current) {
    if (!omega && (rc = ensure_w64(st)) != CONCORD_OK) return rc;
    CK(launch_convert(omega ? st->Om64 : st->W64, 0, ld, out, f32, ld_out, p, p, st->stream));
  } else {
    CK(launch_convert(omega ? st->Om : st->W, 1, ld, out, f32, ld_out, p, p, st->stream));
    if (omega && !f32)
      CK(cudaMemcpy2DAsync(out, (size_t)(ld_out + 1) * sizeof(double), st->omdiag64, sizeof(double),
                           sizeof(double), p, cudaMemcpyDeviceToDevice, st->stream));
  }
  CK(cudaStreamSynchronize(st->stream));
  return CONCORD_OK;
}

int concord_get_omega(concord_state* st, void* Om_dev, int dtype, int ld) {
  return get_matrix(st, true, Om_dev, dtype, ld);
}

int concord_get_W(concord_state* st, void* W_dev, int dtype, int ld) {
  return get_matrix(st, false, W_dev, dtype, ld);
}

int concord_get_history(concord_state* st, double* hist_host, int max_rows, int* rows) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!rows) return fail(CONCORD_E_ARG, "rows is NULL");
  int n = st->hist_rows < max_rows ? st->hist_rows : max_rows;
  if (n > kHistCap) n = kHistCap;
  if (n > 0 && hist_host)
    CK(cudaMemcpy(hist_host, st->hist, sizeof(double) * kHist * (size_t)n, cudaMemcpyDeviceToHost));
  *rows = st->hist_rows;
  return CONCORD_OK;
}

int concord_get_timing(concord_state* st, double* launch_ms, int* launch_sweeps, int max_launches,
                       int* n_launches) {
  if (!st || !n_launches) return fail(CONCORD_E_ARG, "state and n_launches must be non-NULL");
  const int n = st->n_launch < max_launches ? st->n_launch : max_launches;
  for (int q = 0; q < n; ++q) {
    if (launch_ms) launch_ms[q] = st->launch_ms[q];
    if (launch_sweeps) launch_sweeps[q] = st->launch_sweeps[q];
  }
  *n_launches = st->n_launch;
  return CONCORD_OK;
}

unsigned long long concord_kernel_launches(void) { return launches_so_far(); }

int concord_sweep(concord_state* st, double lambda, int n_sweeps, concord_result* res) {
  int rc = check_state(st);
  if (rc) return rc;
  return run_impl(st, lambda, -1.0, n_sweeps, CONCORD_STOP_KKT, 0.0, 1, res);
}

int concord_run(concord_state* st, double lambda, double tol, int max_sweeps, int stop_rule,
                double switch_tol, concord_result* res) {
  int rc = check_state(st);
  if (rc) return rc;
  return run_impl(st, lambda, tol, max_sweeps, stop_rule, switch_tol, 0, res);
}

static int gram_into_state(concord_state* st, const void* X, int x_f32, int n, int ldx, int prep,
                           double screen_lambda = 0.0);

int concord_path(concord_state* st, const double* lambdas, int n_lambda, double tol,
                 int max_sweeps, concord_result* results, void* omega_out_dev, int ld_out) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!lambdas || n_lambda < 1 || !(tol > 0.0) || max_sweeps < 1 ||
      (omega_out_dev && ld_out < st->p))
    return fail(CONCORD_E_ARG, "lambdas non-NULL, n_lambda >= 1, tol > 0, max_sweeps >= 1, "
                               "ld_out >= p when Omega is requested");
  for (int k = 0; k < n_lambda; ++k)
    if (!(lambdas[k] >= 0.0)) return fail(CONCORD_E_ARG, "lambda[%d] must be >= 0", k);
  if ((rc = ensure_screen(st)) || (rc = ensure_path(st, n_lambda, 0))) return rc;
  CK(cudaMemcpyAsync(st->path_lam, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice,
                     st->stream));
  if (is_mixed(st)) {
    if (st->om64_current && (rc = demote_from_fp64(st)) != CONCORD_OK) return rc;
    st->om64_current = false;
    return path_impl<float>(st, lambdas, n_lambda, tol, max_sweeps, results, omega_out_dev, ld_out,
                            nullptr);
  }
  return path_impl<double>(st, lambdas, n_lambda, tol, max_sweeps, results, omega_out_dev, ld_out,
                           nullptr);
}

// One worker of concord_stability: subsamples b = first, first + stride, ...
// on its own state (own stream and CTA budget), adding support counts into
// the shared frequency buffer.
static int stability_worker(concord_state* st, const void* X_dev, int x_dtype, int ldx, int prep,
                            const int* rows_dev, const size_t* offs, const int* set_sizes,
                            int n_sets, int first, int stride, const double* lambdas, int n_lambda,
                            double tol, int max_sweeps, float* freq_dev, std::string* err) {
  int rc = CONCORD_OK;
  for (int b = first; b < n_sets && rc == CONCORD_OK; b += stride) {
    const int nb = set_sizes[b];
    cudaError_t e = launch_gather_rows(X_dev, x_dtype == CONCORD_F32, ldx, rows_dev + offs[b], nb,
                                       st->p, st->Xstage, st->stream);
    if (e != cudaSuccess) {
      rc = fail(CONCORD_E_CUDA, "gather: %s", cudaGetErrorString(e));
      break;
    }
    if ((rc = gram_into_state(st, st->Xstage, 0, nb, st->p, prep)) != CONCORD_OK) break;
    rc = is_mixed(st) ? path_impl<float>(st, lambdas, n_lambda, tol, max_sweeps, nullptr, nullptr,
                                         0, freq_dev)
                      : path_impl<double>(st, lambdas, n_lambda, tol, max_sweeps, nullptr, nullptr,
                                          0, freq_dev);
  }
  if (rc != CONCORD_OK) *err = g_err;
  return rc;
}

int concord_stability(concord_state* st, const void* X_dev, int x_dtype, int n, int ldx, int prep,
                      const int* rows, const int* set_sizes, int n_sets, const double* lambdas,
                      int n_lambda, double tol, int max_sweeps, int n_workers, float* freq_dev) {
  int rc = check_state(st);
  if (rc) return rc;
  const int p = st->p;
  if (!X_dev || !rows || !set_sizes || n_sets < 1 || !lambdas || n_lambda < 1 || !freq_dev ||
      n < 1 || ldx < p || prep < 0 || prep > 2 || !(tol > 0.0) || max_sweeps < 1 ||
      n_workers < 0 || (x_dtype != CONCORD_F64 && x_dtype != CONCORD_F32))
    return fail(CONCORD_E_ARG, "bad argument to concord_stability");
  const bool batched = n_workers == 0;
  if (n_workers > n_sets) n_workers = n_sets;
  if (n_workers > st->sms) n_workers = st->sms;
  size_t total = 0;
  for (int b = 0; b < n_sets; ++b) {
    if (set_sizes[b] < 2 || set_sizes[b] > st->n_cap)
      return fail(CONCORD_E_ARG, "subsample %d: size must be in 2..n_cap (%d)", b, st->n_cap);
    total += (size_t)set_sizes[b];
  }
  for (size_t q = 0; q < total; ++q)
    if (rows[q] < 0 || rows[q] >= n) return fail(CONCORD_E_ARG, "row index out of range");
  for (int k = 0; k < n_lambda; ++k)
    if (!(lambdas[k] >= 0.0)) return fail(CONCORD_E_ARG, "lambda[%d] must be >= 0", k);
  if ((rc = ensure_screen(st)) || (rc = ensure_path(st, n_lambda, total))) return rc;
  CK(cudaMemcpyAsync(st->path_lam, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice,
                     st->stream));
  CK(cudaMemcpyAsync(st->rows_dev, rows, sizeof(int) * total, cudaMemcpyHostToDevice, st->stream));
  CK(cudaMemsetAsync(freq_dev, 0, sizeof(float) * (size_t)n_lambda * p * p, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  std::vector<size_t> offs(n_sets);
  for (int b = 0, o = 0; b < n_sets; o += set_sizes[b], ++b) offs[b] = (size_t)o;
  if (batched) {
    // every subsample one problem of a batch: one persistent launch per wave
    // of co-resident problems (concord_batch_*), support counts added by the
    // kernel after each lambda
    int n_max = 2;
    for (int b = 0; b < n_sets; ++b) n_max = set_sizes[b] > n_max ? set_sizes[b] : n_max;
    std::vector<int> ps(n_sets, p);
    concord_batch* bt = nullptr;
    rc = concord_batch_create(&bt, n_sets, ps.data(), st->precision, n_max, st->device);
    if (rc != CONCORD_OK) return rc;
    concord_batch_set_stream(bt, st->stream);
    concord_batch_set_timeout(bt, st->timeout_s);
    for (int b = 0; b < n_sets && rc == CONCORD_OK; ++b)
      rc = concord_batch_gram(bt, b, X_dev, x_dtype, n, ldx, st->rows_dev + offs[b], set_sizes[b],
                              prep);
    if (rc == CONCORD_OK)
      rc = concord_batch_path(bt, lambdas, n_lambda, tol, max_sweeps, nullptr, freq_dev);
    if (rc == CONCORD_OK) concord_batch_info(bt, &st->last_batch_rows, nullptr, nullptr, nullptr);
    concord_batch_destroy(bt);
    if (rc != CONCORD_OK) return rc;
  } else if (n_workers <= 1) {
    std::string err;
    rc = stability_worker(st, X_dev, x_dtype, ldx, prep, st->rows_dev, offs.data(), set_sizes,
                          n_sets, 0, 1, lambdas, n_lambda, tol, max_sweeps, freq_dev, &err);
    if (rc != CONCORD_OK) return rc;
  } else {
    // independent subsamples run concurrently: one state per worker (own
    // stream, 1 / n_workers of the SMs), one host thread each
    std::vector<concord_state*> ws(n_workers, nullptr);
    for (int k = 0; k < n_workers && rc == CONCORD_OK; ++k) {
      rc = concord_create(&ws[k], p, st->precision, st->n_cap, st->device);
      if (rc == CONCORD_OK) {
        ws[k]->gram_mode = st->gram_mode;
        ws[k]->max_ctas = st->sms / n_workers > 0 ? st->sms / n_workers : 1;
        rc = ensure_screen(ws[k]);
        if (rc == CONCORD_OK) rc = ensure_path(ws[k], n_lambda, 0);
        if (rc == CONCORD_OK &&
            cudaMemcpy(ws[k]->path_lam, lambdas, sizeof(double) * n_lambda,
                       cudaMemcpyHostToDevice) != cudaSuccess)
          rc = fail(CONCORD_E_CUDA, "copy of the lambdas failed");
      }
    }
    if (rc == CONCORD_OK) {
      std::vector<int> rcs(n_workers, CONCORD_OK);
      std::vector<std::string> errs(n_workers);
      std::vector<std::thread> th;
      for (int k = 0; k < n_workers; ++k)
        th.emplace_back([&, k]() {
          cudaSetDevice(st->device);
          rcs[k] = stability_worker(ws[k], X_dev, x_dtype, ldx, prep, st->rows_dev, offs.data(),
                                    set_sizes, n_sets, k, n_workers, lambdas, n_lambda, tol,
                                    max_sweeps, freq_dev, &errs[k]);
        });
      for (auto& t : th) t.join();
      for (int k = 0; k < n_workers; ++k)
        if (rcs[k] != CONCORD_OK && rc == CONCORD_OK) {
          rc = rcs[k];
          g_err = errs[k];
        }
    }
    for (auto* w : ws)
      if (w) concord_destroy(w);
    if (rc != CONCORD_OK) return rc;
  }
  CK(launch_scale_f32(freq_dev, (size_t)n_lambda * p * p, 1.0f / n_sets, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  return CONCORD_OK;
}

int concord_set_poll_sleep(concord_state* st, int ns) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (ns > 100000) return fail(CONCORD_E_ARG, "poll sleep must be <= 100000 ns");
  st->poll_ns = ns < 0 ? -1 : ns;
  return CONCORD_OK;
}

int concord_set_sweep_variant(concord_state* st, int variant) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (variant < 0 || variant > 4) return fail(CONCORD_E_ARG, "variant must be 0..4 (CONCORD_SWEEP_*)");
  st->sweep_variant = variant;
  return CONCORD_OK;
}

int concord_autotune(concord_state* st, double lambda, double tol, int max_sweeps,
                     double* ms_per_sweep, int* variant, int* rows_per_warp) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!(lambda >= 0.0) || !(tol > 0.0) || max_sweeps < 1)
    return fail(CONCORD_E_ARG, "lambda >= 0, tol > 0, max_sweeps >= 1 required");
  // screened; dense cluster and grid layouts at 32, 16, 8, 4 rows per warp
  struct Choice { int variant, rows; };
  const Choice choices[kAutotuneChoices] = {
      {CONCORD_SWEEP_SCREENED, 0}, {CONCORD_SWEEP_CLUSTER, 32}, {CONCORD_SWEEP_CLUSTER, 16},
      {CONCORD_SWEEP_CLUSTER, 8},  {CONCORD_SWEEP_CLUSTER, 4},  {CONCORD_SWEEP_GRID, 32},
      {CONCORD_SWEEP_GRID, 16},    {CONCORD_SWEEP_GRID, 8},     {CONCORD_SWEEP_GRID, 4}};
  const int keep_variant = st->sweep_variant, keep_rows = st->rows_per_warp;
  int best = -1;
  double best_ms = 0.0;
  for (int c = 0; c < kAutotuneChoices; ++c) {
    if (ms_per_sweep) ms_per_sweep[c] = -1.0;
    st->sweep_variant = choices[c].variant;
    st->rows_per_warp = choices[c].rows;
    if ((rc = reset_iterate(st)) != CONCORD_OK) break;
    concord_result r;
    rc = run_impl(st, lambda, tol, max_sweeps, CONCORD_STOP_KKT, 0.0, 0, &r);
    if (rc == CONCORD_E_ARG || rc == CONCORD_E_OCCUPANCY) {  // layout not launchable here
      rc = CONCORD_OK;
      continue;
    }
    if (rc != CONCORD_OK && rc != CONCORD_NOT_CONVERGED) break;
    rc = CONCORD_OK;
    double ms = 0.0;
    int sw = 0;
    for (int q = 0; q < st->n_launch; ++q) {
      ms += st->launch_ms[q];
      sw += st->launch_sweeps[q];
    }
    const double per = ms / (sw > 0 ? sw : 1);
    if (ms_per_sweep) ms_per_sweep[c] = per;
    if (best < 0 || per < best_ms) {
      best = c;
      best_ms = per;
    }
  }
  if (rc != CONCORD_OK || best < 0) {
    st->sweep_variant = keep_variant;
    st->rows_per_warp = keep_rows;
    if (rc == CONCORD_OK) rc = fail(CONCORD_E_OCCUPANCY, "no sweep layout could run");
    reset_iterate(st);
    return rc;
  }
  st->sweep_variant = choices[best].variant;
  st->rows_per_warp = choices[best].rows;
  if (variant) *variant = choices[best].variant;
  if (rows_per_warp) *rows_per_warp = choices[best].rows;
  return reset_iterate(st);
}

int concord_get_sweep_variant(concord_state* st, int* variant, int* cluster_size) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (variant) *variant = st->last_variant;
  if (cluster_size) *cluster_size = st->cluster_size;
  return CONCORD_OK;
}

int concord_set_rows_per_warp(concord_state* st, int rows) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (rows < 0 || rows > 32) return fail(CONCORD_E_ARG, "rows per warp must be in 0..32");
  st->rows_per_warp = rows;
  return CONCORD_OK;
}

int concord_set_lazy_verify(concord_state* st, int on) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (on != 0 && on != 1) return fail(CONCORD_E_ARG, "on must be 0 or 1");
  st->lazy_verify = on == 1;
  return CONCORD_OK;
}

int concord_set_sparse_polish(concord_state* st, int on) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (on != 0 && on != 1) return fail(CONCORD_E_ARG, "on must be 0 or 1");
  st->sparse_polish = on == 1;
  return CONCORD_OK;
}

int concord_set_refine(concord_state* st, int on) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (on != 0 && on != 1) return fail(CONCORD_E_ARG, "on must be 0 or 1");
  st->refine = on == 1;
  return CONCORD_OK;
}

int concord_set_gram_mode(concord_state* st, int mode) {
  if (!st) return fail(CONCORD_E_ARG, "state is NULL");
  if (mode != CONCORD_GRAM_FP64 && mode != CONCORD_GRAM_FP32 && mode != CONCORD_GRAM_TF32X3 &&
      mode != CONCORD_GRAM_BF16X3)
    return fail(CONCORD_E_ARG, "unknown Gram mode %d", mode);
  if ((mode == CONCORD_GRAM_TF32X3 || mode == CONCORD_GRAM_BF16X3) && !is_mixed(st))
    return fail(CONCORD_E_ARG, "the tensor-core Gram feeds the mixed-precision state only");
  st->gram_mode = mode;
  return CONCORD_OK;
}

// X (device) -> S in the state, per the state's Gram mode.
static int gram_into_state(concord_state* st, const void* X, int x_f32, int n, int ldx, int prep,
                           double screen_lambda) {
  st->prescreen = false;
  const int p = st->p, ld = st->ld;
  CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  // the FP64 W (free until the iterate is reset below) holds the column partials
  CK(launch_col_stats_chunked(X, x_f32, n, p, ldx, prep, st->mean, st->inv_scale, st->flag,
                              st->W64, st->stream));
  // the reduced-precision Grams keep the FP32 data (transposed) for the S
  // refinement of a later polish; the FP64 Gram is exact already
  st->zt_valid = false;
  st->zt_n = n;
  st->zt_ldn = round_up(n, 32);
  float* zt = (st->zt32 && is_mixed(st)) ? st->zt32 : nullptr;
  switch (st->gram_mode) {
    case CONCORD_GRAM_FP64:
      if (is_mixed(st)) {
        // FP64 Gram for a mixed state: Z in the FP32 workspace is too narrow,
        // so stage Z in W64 (free until polishing) when it fits
        if ((size_t)n * ld > (size_t)p * ld) return fail(CONCORD_E_ARG, "FP64 Gram for mixed state needs n <= p");
        CK(launch_apply_prep(X, x_f32, n, p, ldx, st->mean, st->inv_scale, st->W64, 0, ld, st->stream));
        CK(launch_syrk_f64(st->W64, n, p, ld, st->S64, ld, 1.0 / n, st->stream));
        CK(launch_convert(st->S64, 0, ld, st->S, 1, ld, p, p, st->stream));
      } else {
        CK(launch_apply_prep(X, x_f32, n, p, ldx, st->mean, st->inv_scale, st->Z, 0, st->ldz,
                             st->stream));
        CK(launch_syrk_f64((const double*)st->Z, n, p, st->ldz, st->S64, ld, 1.0 / n, st->stream));
      }
      break;
    case CONCORD_GRAM_FP32: {
      float* Zf = (float*)st->Z;
      if (!is_mixed(st)) return fail(CONCORD_E_ARG, "FP32 Gram feeds the mixed state only");
      CK(launch_apply_prep(X, x_f32, n, p, ldx, st->mean, st->inv_scale, Zf, 1, st->ldz, st->stream));
      CK(launch_syrk_f32(Zf, n, p, st->ldz, (float*)st->S, ld, 1.0f / n, st->stream));
      if (zt) {
        CK(launch_split_tf32(X, x_f32, n, p, ldx, st->mean, st->inv_scale, nullptr, nullptr,
                             st->zt_ldn, st->p_pad, st->stream, zt, st->zt_ldn));
        st->zt_valid = true;
      }
      break;
    }
    case CONCORD_GRAM_TF32X3: {
      CK(launch_split_tf32(X, x_f32, n, p, ldx, st->mean, st->inv_scale, st->zt_hi, st->zt_lo,
                           round_up(n, 32), st->p_pad, st->stream, zt, st->zt_ldn));
      st->zt_valid = zt != nullptr;
      cudaError_t e = launch_gram_tf32x3(st->zt_hi, st->zt_lo, round_up(n, 32), st->p_pad, p,
                                         (float*)st->S, ld, 1.0f / n, st->flag, st->stream);
      if (e == cudaErrorNotSupported) return fail(CONCORD_E_CUDA, "tensor-core Gram unavailable");
      CK(e);
      break;
    }
    case CONCORD_GRAM_BF16X3: {
      uint16_t* hi = (uint16_t*)st->zt_hi;
      uint16_t* lo = (uint16_t*)st->zt_lo;
      CK(launch_split_bf16(X, x_f32, n, p, ldx, st->mean, st->inv_scale, hi, lo, round_up(n, 64),
                           st->p_pad, st->stream, zt, st->zt_ldn));
      st->zt_valid = zt != nullptr;
      cudaError_t e = launch_gram_bf16x3(hi, lo, round_up(n, 64), st->p_pad, p, (float*)st->S, ld,
                                         1.0f / n, st->flag, st->stream);
      if (e == cudaErrorNotSupported) return fail(CONCORD_E_CUDA, "tensor-core Gram unavailable");
      CK(e);
      break;
    }
    default:
      return fail(CONCORD_E_ARG, "unknown Gram mode");
  }
  // mixed state from an FP32 S: the FP64 copy and the starting iterate in
  // one pass over S (checks in bits 8 and 16 of the same flag, one read)
  const bool fused = is_mixed(st) && st->gram_mode != CONCORD_GRAM_FP64;
  bool screened_start = false;
  if (fused) {
    ResetMixedArgs ra;
    ra.S = (const float*)st->S;
    ra.ld = ld;
    ra.p = p;
    ra.P = st->P;
    ra.W = (float*)st->W;
    ra.Om = (float*)st->Om;
    ra.S64 = st->S64;
    ra.mrow = st->mrow;
    ra.sdiag64 = st->sdiag64;
    ra.sdiag32 = (float*)st->sdiagT;
    ra.sd1 = (float*)st->sd1;
    ra.sd2 = (float*)st->sd2;
    ra.sd1_64 = st->sd1_64;
    ra.sd2_64 = st->sd2_64;
    ra.omdiag64 = st->omdiag64;
    ra.bad = st->flag;
    ra.lam_s = 0.f;
    // the start screen of the coming solve (the screened kernel's own
    // predicate on W = S, Omega = I), when its lambda is known and the solve
    // will take the screened kernel
    const int sv = st->sweep_variant;
    if (screen_lambda > 0.0 && st->fault_vertex < 0 &&
        (sv == CONCORD_SWEEP_AUTO || sv == CONCORD_SWEEP_SCREENED)) {
      int rc2 = ensure_screen(st);
      if (rc2 != CONCORD_OK) return rc2;
      const ScreenLayout L = screen_layout(p, st->P, st->nc_cap, st->term_cap);
      CK(cudaMemsetAsync((char*)st->scr + L.ctr, 0, sizeof(int) * kCtrs, st->stream));
      CK(cudaMemsetAsync((char*)st->scr + L.cnt_r0, 0, sizeof(int) * (size_t)(p + 1), st->stream));
      CK(cudaMemsetAsync((char*)st->scr + L.cnt_r1, 0, sizeof(int) * (size_t)(p + 1), st->stream));
      const ScreenWork<float> sw = screen_work<float>(st);
      ra.lam_s = (float)(screen_lambda * (1.0 - kScreenMargin));
      ra.cand = sw.cand[0];
      ra.n_cand = sw.ctr + kCtrCand;
      ra.cnt_r = sw.cnt_r[0];
      ra.nc_cap = st->nc_cap;
      screened_start = true;
    }
    CK(launch_reset_mixed(ra, st->stream));
  }
  st->om64_current = false;
  if (screened_start) {
    // the solve's screened launch comes next: it reads the checks' word on
    // the device and the host reads it with the launch's result (no wait here)
    st->prescreen = true;
    st->prescreen_lambda = screen_lambda;
    st->flag_pending = true;
    return CONCORD_OK;
  }
  int bad = 0, rc;
  if ((rc = read_flag(st, &bad))) return rc;
  if ((bad & 7) || !fused) {
    if ((rc = input_flag_error(bad & 7))) return rc;
    return reset_iterate(st);
  }
  return input_flag_error(bad);
}

int concord_gram(const void* X_dev, int x_dtype, int n, int p, int ldx, int prep, int mode,
                 void* S_dev, int s_dtype, int lds, void* stream) {
  if (!X_dev || !S_dev || n < 1 || p < 2 || ldx < p || lds < p)
    return fail(CONCORD_E_ARG, "X/S non-NULL, n >= 1, p >= 2, ldx >= p, lds >= p required");
  if ((x_dtype != CONCORD_F64 && x_dtype != CONCORD_F32) ||
      (s_dtype != CONCORD_F64 && s_dtype != CONCORD_F32) || prep < 0 || prep > 2)
    return fail(CONCORD_E_ARG, "bad dtype or prep");
  cudaStream_t s = (cudaStream_t)stream;
  const int x_f32 = x_dtype == CONCORD_F32, s_f32 = s_dtype == CONCORD_F32;
  const int ld = round_up(p, kTile);
  double *mean = nullptr, *inv = nullptr, *part = nullptr;
  int* bad = nullptr;
  void* Z = nullptr;
  void* Sw = nullptr;
  float *hi = nullptr, *lo = nullptr;
  int rc = CONCORD_OK, hbad = 0;
  cudaError_t e = cudaSuccess;
#define GK(expr)                                                                   \
  do {                                                                             \
    e = (expr);                                                                    \
    if (e != cudaSuccess) {                                                        \
      rc = fail(e == cudaErrorMemoryAllocation ? CONCORD_E_NOMEM : CONCORD_E_CUDA, \
                "%s: %s", #expr, cudaGetErrorString(e));                           \
      goto done;                                                                   \
    }                                                                              \
  } while (0)
  GK(cudaMallocAsync((void**)&mean, sizeof(double) * p, s));
  GK(cudaMallocAsync((void**)&inv, sizeof(double) * p, s));
  GK(cudaMallocAsync((void**)&bad, sizeof(int), s));
  GK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  GK(cudaMallocAsync((void**)&part, sizeof(double) * (size_t)col_stats_chunks(n) * p, s));
  GK(launch_col_stats_chunked(X_dev, x_f32, n, p, ldx, prep, mean, inv, bad, part, s));
  if (mode == CONCORD_GRAM_FP64) {
    GK(cudaMallocAsync(&Z, sizeof(double) * (size_t)n * ld, s));
    GK(launch_apply_prep(X_dev, x_f32, n, p, ldx, mean, inv, Z, 0, ld, s));
    if (s_f32) {
      GK(cudaMallocAsync(&Sw, sizeof(double) * (size_t)p * ld, s));
      GK(launch_syrk_f64((const double*)Z, n, p, ld, (double*)Sw, ld, 1.0 / n, s));
      GK(launch_convert(Sw, 0, ld, S_dev, 1, lds, p, p, s));
    } else {
      GK(launch_syrk_f64((const double*)Z, n, p, ld, (double*)S_dev, lds, 1.0 / n, s));
    }
  } else if (mode == CONCORD_GRAM_FP32) {
    GK(cudaMallocAsync(&Z, sizeof(float) * (size_t)n * ld, s));
    GK(launch_apply_prep(X_dev, x_f32, n, p, ldx, mean, inv, Z, 1, ld, s));
    if (s_f32) {
      GK(launch_syrk_f32((const float*)Z, n, p, ld, (float*)S_dev, lds, 1.0f / n, s));
    } else {
      GK(cudaMallocAsync(&Sw, sizeof(float) * (size_t)p * ld, s));
      GK(launch_syrk_f32((const float*)Z, n, p, ld, (float*)Sw, ld, 1.0f / n, s));
      GK(launch_convert(Sw, 1, ld, S_dev, 0, lds, p, p, s));
    }
  } else if (mode == CONCORD_GRAM_TF32X3 || mode == CONCORD_GRAM_BF16X3) {
    const bool bf = mode == CONCORD_GRAM_BF16X3;
    const int n_pad = round_up(n, bf ? 64 : 32), p_pad = round_up(p, 128);
    const size_t esz = bf ? 2 : 4;
    GK(cudaMallocAsync((void**)&hi, esz * (size_t)n_pad * p_pad, s));
    GK(cudaMallocAsync((void**)&lo, esz * (size_t)n_pad * p_pad, s));
    if (bf)
      GK(launch_split_bf16(X_dev, x_f32, n, p, ldx, mean, inv, (uint16_t*)hi, (uint16_t*)lo, n_pad,
                           p_pad, s));
    else
      GK(launch_split_tf32(X_dev, x_f32, n, p, ldx, mean, inv, hi, lo, n_pad, p_pad, s));
    float* Sout = (float*)S_dev;
    int ldo = lds;
    if (!s_f32) {
      GK(cudaMallocAsync(&Sw, sizeof(float) * (size_t)p * ld, s));
      Sout = (float*)Sw;
      ldo = ld;
    }
    e = bf ? launch_gram_bf16x3((const uint16_t*)hi, (const uint16_t*)lo, n_pad, p_pad, p, Sout, ldo,
                                1.0f / n, bad, s)
           : launch_gram_tf32x3(hi, lo, n_pad, p_pad, p, Sout, ldo, 1.0f / n, bad, s);
    if (e == cudaErrorNotSupported) {
      rc = fail(CONCORD_E_CUDA, "tensor-core Gram unavailable on this device");
      goto done;
    }
    GK(e);
    if (!s_f32) GK(launch_convert(Sw, 1, ld, S_dev, 0, lds, p, p, s));
  } else {
    rc = fail(CONCORD_E_ARG, "unknown Gram mode %d", mode);
    goto done;
  }
  GK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GK(cudaStreamSynchronize(s));
  if (hbad & 4) rc = fail(CONCORD_E_TIMEOUT, "tensor-core Gram: a device-side wait ran out");
  else if (hbad & 2) rc = fail(CONCORD_E_NONFINITE, "X has a non-finite entry");
  else if (hbad & 1 && prep == CONCORD_PREP_STANDARDIZE)
    rc = fail(CONCORD_E_NONPOS_DIAG, "X has a constant column");
done:
  if (mean) cudaFreeAsync(mean, s);
  if (part) cudaFreeAsync(part, s);
  if (inv) cudaFreeAsync(inv, s);
  if (bad) cudaFreeAsync(bad, s);
  if (Z) cudaFreeAsync(Z, s);
  if (Sw) cudaFreeAsync(Sw, s);
  if (hi) cudaFreeAsync(hi, s);
  if (lo) cudaFreeAsync(lo, s);
#undef GK
  return rc;
}

int concord_solve_device(concord_state* st, const void* X_dev, int x_dtype, int n, int ldx,
                         int prep, double lambda, double tol, int max_sweeps, int stop_rule,
                         void* Omega_dev, int omega_dtype, int ldo, concord_result* res) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!X_dev || n < 1 || n > st->n_cap || ldx < st->p || prep < 0 || prep > 2 ||
      (x_dtype != CONCORD_F64 && x_dtype != CONCORD_F32))
    return fail(CONCORD_E_ARG, "X_dev non-NULL, 1 <= n <= n_cap (%d), ldx >= p, prep in 0..2",
                st->n_cap);
  cudaEvent_t e0;
  CK(cudaEventCreate(&e0));
  CK(cudaEventRecord(e0, st->stream));
  rc = gram_into_state(st, X_dev, x_dtype == CONCORD_F32, n, ldx, prep, lambda);
  if (rc == CONCORD_OK) {
    concord_result r;
    rc = run_impl(st, lambda, tol, max_sweeps, stop_rule, 0.0, 0, &r);
    if ((rc == CONCORD_OK || rc == CONCORD_NOT_CONVERGED) && Omega_dev) {
      int rc2 = get_matrix(st, true, Omega_dev, omega_dtype, ldo);
      if (rc2 != CONCORD_OK) rc = rc2;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, st->ev1);
    r.seconds = ms * 1e-3;
    if (res) *res = r;
  }
  cudaEventDestroy(e0);
  return rc;
}

int concord_solve_host(concord_state* st, const double* X_host, int n, int prep, double lambda,
                       double tol, int max_sweeps, int stop_rule, double* Omega_host,
                       concord_result* res) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!X_host || n < 1 || n > st->n_cap) return fail(CONCORD_E_ARG, "X_host non-NULL, 1 <= n <= n_cap");
  const int p = st->p;
  CK(cudaMemcpyAsync(st->Xstage, X_host, sizeof(double) * (size_t)n * p, cudaMemcpyHostToDevice,
                     st->stream));
  rc = concord_solve_device(st, st->Xstage, CONCORD_F64, n, p, prep, lambda, tol, max_sweeps,
                            stop_rule, nullptr, CONCORD_F64, p, res);
  if ((rc == CONCORD_OK || rc == CONCORD_NOT_CONVERGED) && Omega_host) {
    const double* src = (!is_mixed(st) || st->om64_current) ? st->Om64 : nullptr;
    if (!src) return fail(CONCORD_E_CUDA, "no FP64 iterate to copy out");
    CK(cudaMemcpy2DAsync(Omega_host, sizeof(double) * p, src, sizeof(double) * st->ld,
                         sizeof(double) * p, p, cudaMemcpyDeviceToHost, st->stream));
    CK(cudaStreamSynchronize(st->stream));
  }
  return rc;
}

int concord_solve(const double* data_host, int is_X, int n, int p, int prep, double lambda,
                  double tol, int max_sweeps, int precision, const double* Omega0_host,
                  double* Omega_host, concord_result* res) {
  if (!data_host || p < 2 || (is_X && n < 1)) return fail(CONCORD_E_ARG, "data non-NULL, p >= 2, n >= 1");
  concord_state* st = nullptr;
  int rc = concord_create(&st, p, precision, is_X ? n : 0, -1);
  if (rc) return rc;
  double* tmp = nullptr;
  if (is_X) {
    if (Omega0_host) {
      concord_destroy(st);
      return fail(CONCORD_E_ARG, "a warm start needs S input (is_X = 0)");
    }
    rc = concord_solve_host(st, data_host, n, prep, lambda, tol, max_sweeps, CONCORD_STOP_KKT,
                            Omega_host, res);
  } else {
    if (cudaMalloc((void**)&tmp, sizeof(double) * (size_t)p * p) != cudaSuccess) {
      concord_destroy(st);
      return fail(CONCORD_E_NOMEM, "cudaMalloc for S");
    }
    rc = CONCORD_OK;
    if (cudaMemcpy(tmp, data_host, sizeof(double) * (size_t)p * p, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(CONCORD_E_CUDA, "copy of S failed");
    if (rc == CONCORD_OK) rc = concord_set_S(st, tmp, CONCORD_F64, p);
    if (rc == CONCORD_OK && Omega0_host) {
      if (cudaMemcpy(tmp, Omega0_host, sizeof(double) * (size_t)p * p, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(CONCORD_E_CUDA, "copy of Omega0 failed");
      if (rc == CONCORD_OK) rc = concord_set_omega(st, tmp, CONCORD_F64, p);
    }
    if (rc == CONCORD_OK) rc = concord_run(st, lambda, tol, max_sweeps, CONCORD_STOP_KKT, 0.0, res);
    if ((rc == CONCORD_OK || rc == CONCORD_NOT_CONVERGED) && Omega_host) {
      int rc2 = concord_get_omega(st, tmp, CONCORD_F64, p);
      if (rc2 == CONCORD_OK &&
          cudaMemcpy(Omega_host, tmp, sizeof(double) * (size_t)p * p, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc2 = fail(CONCORD_E_CUDA, "copy of Omega failed");
      if (rc2 != CONCORD_OK) rc = rc2;
    }
    cudaFree(tmp);
  }
  concord_destroy(st);
  return rc;
}

int concord_lambda_max(concord_state* st, double* lambda_max) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!lambda_max) return fail(CONCORD_E_ARG, "lambda_max is NULL");
  CK(cudaMemsetAsync(st->lmax, 0, sizeof(unsigned long long), st->stream));
  CK(launch_lambda_max(st->S64, st->p, st->ld, st->lmax, st->stream));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(st->h_result, st->lmax, sizeof bits, cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  memcpy(&bits, st->h_result, sizeof bits);
  memcpy(lambda_max, &bits, sizeof bits);
  return CONCORD_OK;
}

// ------------------------------------------------------- implicit differentiation

static int adj_alloc(concord_state* st, void** ptr, size_t bytes) {
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  CK(cudaMalloc(ptr, bytes));
  return CONCORD_OK;
}

// CSR of the active set of the current Omega (FP64 copy when it holds the
// iterate), its mirror map and the Jacobi preconditioner.
static int adj_build(concord_state* st) {
  auto& A = st->adj;
  const int p = st->p;
  int rc;
  if (!A.rowptr) {
    if ((rc = adj_alloc(st, (void**)&A.cnt, sizeof(int) * p)) ||
        (rc = adj_alloc(st, (void**)&A.rowptr, sizeof(int) * (p + 1))) ||
        (rc = adj_alloc(st, (void**)&A.bad, sizeof(int))) ||
        (rc = adj_alloc(st, (void**)&A.scal, sizeof(double) * (kAdjRes + 2))))
      return rc;
  }
  const bool f64 = !is_mixed(st) || st->om64_current;
  const void* Om = f64 ? (const void*)st->Om64 : st->Om;
  const int f32 = f64 ? 0 : 1;
  CK(launch_adj_count(Om, f32, p, st->ld, A.cnt, st->sms, st->stream));
  CK(launch_adj_scan(A.cnt, p, A.rowptr, st->stream));
  int nnz = 0;
  CK(cudaMemcpyAsync(st->h_flag, A.rowptr + p, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  nnz = *st->h_flag;
  if (nnz > A.cap) {
    const size_t n = (size_t)nnz;
    int** ints[] = {&A.col, &A.erow, &A.mirror};
    for (int** q : ints)
      if ((rc = adj_alloc(st, (void**)q, sizeof(int) * n))) return rc;
    double** dbl[] = {&A.om, &A.minv, &A.b, &A.x, &A.r, &A.z, &A.p0, &A.p1, &A.q};
    for (double** q : dbl)
      if ((rc = adj_alloc(st, (void**)q, sizeof(double) * n))) return rc;
    A.cap = nnz;
  }
  A.nnz = nnz;
  A.rhs_ready = false;
  A.solved = false;
  CK(cudaMemsetAsync(A.bad, 0, sizeof(int), st->stream));
  CK(launch_adj_fill(Om, f32, p, st->ld, A.rowptr, A.col, A.erow, A.om, st->sms, st->stream));
  CK(launch_adj_prep(nnz, A.rowptr, A.col, A.erow, A.om, st->sdiag64, A.mirror, A.minv, A.bad,
                     st->sms, st->stream));
  CK(cudaMemcpyAsync(st->h_flag, A.bad, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  if (*st->h_flag)
    return fail(CONCORD_E_ARG, "Omega is not symmetric or has a non-positive diagonal");
  return CONCORD_OK;
}

static bool dtype_ok(int t) { return t == CONCORD_F64 || t == CONCORD_F32; }

int concord_heldout(concord_state* st, const void* Sval_dev, int s_dtype, int lds, double* loss_host) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!Sval_dev || !loss_host || lds < st->p || !dtype_ok(s_dtype))
    return fail(CONCORD_E_ARG, "S_val and loss must be non-NULL, lds >= p, s_dtype F64 or F32");
  if ((rc = adj_build(st))) return rc;
  auto& A = st->adj;
  // the per-CTA loss partials use the iteration vector r as scratch
  CK(launch_adj_heldout(A.nnz, A.rowptr, A.col, A.erow, A.mirror, A.om, Sval_dev,
                        s_dtype == CONCORD_F32, lds, A.b, A.r, A.cap, A.scal + kAdjRes, st->sms,
                        st->stream));
  CK(cudaMemcpyAsync(st->h_result, A.scal + kAdjRes, sizeof(double), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  *loss_host = st->h_result[0];
  A.rhs_ready = true;
  if (!isfinite(*loss_host)) return fail(CONCORD_E_NONFINITE, "held-out loss is not finite");
  return CONCORD_OK;
}

int concord_adjoint(concord_state* st, const void* gOmega_dev, int g_dtype, int ldg, double tol,
                    int max_iter, double* dS_dev, int ldds, concord_adjoint_info* info) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!info || !(tol > 0.0) || max_iter < 1 || (dS_dev && ldds < st->p) ||
      (gOmega_dev && (ldg < st->p || !dtype_ok(g_dtype))))
    return fail(CONCORD_E_ARG, "info non-NULL, tol > 0, max_iter >= 1, ldg / ldds >= p");
  auto& A = st->adj;
  if (gOmega_dev) {
    if ((rc = adj_build(st))) return rc;
    CK(launch_adj_rhs_dense(gOmega_dev, g_dtype == CONCORD_F32, ldg, A.nnz, A.col, A.erow, A.b,
                            st->sms, st->stream));
  } else if (!A.rhs_ready) {
    return fail(CONCORD_E_ARG, "gOmega is NULL and no concord_heldout gradient is held");
  }
  int occ = 0;
  CK(adj_cg_occupancy(&occ));
  if (occ < 1) return fail(CONCORD_E_OCCUPANCY, "adjoint kernel cannot be resident");
  int grid = st->sms * (occ < 2 ? occ : 2);
  if (grid > st->max_grid) grid = st->max_grid;
  if (st->max_ctas > 0 && grid > st->max_ctas) grid = st->max_ctas;
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.p = st->p;
  a.ld = st->ld;
  a.nnz = A.nnz;
  a.rowptr = A.rowptr;
  a.col = A.col;
  a.erow = A.erow;
  a.mirror = A.mirror;
  a.om = A.om;
  a.S = st->S64;
  a.minv = A.minv;
  a.b = A.b;
  a.x = A.x;
  a.r = A.r;
  a.z = A.z;
  a.pb0 = A.p0;
  a.pb1 = A.p1;
  a.q = A.q;
  a.partials = st->partials;
  a.barrier = st->barrier;
  a.wait.abort = st->abort_info;
  a.wait.info = st->abort_info + 1;
  a.wait.timeout_ns = (uint64_t)(st->timeout_s * 1e9);
  a.tol = tol;
  a.max_iter = max_iter;
  a.result = A.scal;
  CK(cudaMemsetAsync(st->barrier, 0, sizeof(unsigned), st->stream));
  CK(cudaMemsetAsync(st->abort_info, 0, 3 * sizeof(int), st->stream));
  CK(cudaEventRecord(st->ev0, st->stream));
  CK(launch_adj_cg(a, grid, st->stream));
  CK(cudaEventRecord(st->ev1, st->stream));
  if (dS_dev) CK(launch_adj_dS(st->p, A.rowptr, A.col, A.om, A.x, dS_dev, ldds, st->sms, st->stream));
  CK(cudaMemcpyAsync(st->h_result, A.scal, kAdjRes * sizeof(double), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaMemcpyAsync(st->h_abort, st->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
  const double* r = st->h_result;
  memset(info, 0, sizeof *info);
  info->iterations = (int)r[kAdjIters];
  info->residual = r[kAdjTrue];
  info->dlambda = r[kAdjDlam];
  info->active_pairs = (A.nnz - st->p) / 2;
  info->seconds = ms * 1e-3;
  if (st->h_abort[0] != 0) {
    info->status = CONCORD_E_TIMEOUT;
    return fail(CONCORD_E_TIMEOUT, "device wait ran out in the adjoint (phase %d)", st->h_abort[2]);
  }
  const int code = (int)r[kAdjStatus];
  if (code == 2 || !isfinite(info->dlambda)) {
    info->status = CONCORD_E_NONFINITE;
    return fail(CONCORD_E_NONFINITE, "conjugate gradients broke down after %d iterations",
                info->iterations);
  }
  info->status = code == 0 ? CONCORD_OK : CONCORD_NOT_CONVERGED;
  A.solved = true;
  return CONCORD_OK;
}

int concord_adjoint_data(concord_state* st, const void* X_dev, int x_dtype, int n, int ldx, int prep,
                         void* dX_dev, int dx_dtype, int lddx) {
  int rc = check_state(st);
  if (rc) return rc;
  const int p = st->p;
  auto& A = st->adj;
  if (!X_dev || !dX_dev || n < 1 || ldx < p || lddx < p || !dtype_ok(x_dtype) ||
      !dtype_ok(dx_dtype) || prep < CONCORD_PREP_NONE || prep > CONCORD_PREP_STANDARDIZE)
    return fail(CONCORD_E_ARG, "X and dX non-NULL, n >= 1, ldx / lddx >= p, valid dtypes and prep");
  if (!A.solved) return fail(CONCORD_E_ARG, "no adjoint held: call concord_adjoint first");
  const size_t mat = (size_t)n * st->ld;
  if (n > A.n_cap) {
    double** big[] = {&A.Z, &A.P, &A.Q, &A.dZ};
    for (double** q : big)
      if ((rc = adj_alloc(st, (void**)q, sizeof(double) * mat))) return rc;
    A.n_cap = n;
  }
  if (!A.m1) {
    double** small[] = {&A.m1, &A.m2, &A.mean, &A.scale};
    for (double** q : small)
      if ((rc = adj_alloc(st, (void**)q, sizeof(double) * p))) return rc;
    if ((rc = adj_alloc(st, (void**)&A.part1, sizeof(double) * kAdjColChunks * (size_t)p)) ||
        (rc = adj_alloc(st, (void**)&A.part2, sizeof(double) * kAdjColChunks * (size_t)p)))
      return rc;
  }
  const int xf = x_dtype == CONCORD_F32;
  CK(cudaMemsetAsync(A.bad, 0, sizeof(int), st->stream));
  // A.P (n x ld, written later) holds the column partials
  CK(launch_col_stats_chunked(X_dev, xf, n, p, ldx, prep, A.mean, A.scale, A.bad, A.P, st->stream));
  CK(launch_apply_prep(X_dev, xf, n, p, ldx, A.mean, A.scale, A.Z, 0, st->ld, st->stream));
  CK(launch_adj_data(A.Z, A.P, A.Q, A.dZ, st->ld, n, p, prep, A.rowptr, A.col, A.om, A.x, A.scale,
                     A.part1, A.part2, A.m1, A.m2, dX_dev, dx_dtype == CONCORD_F32, lddx, st->sms,
                     st->stream));
  CK(cudaMemcpyAsync(st->h_flag, A.bad, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  if (*st->h_flag & 2) return fail(CONCORD_E_NONFINITE, "non-finite value in X");
  if (*st->h_flag) return fail(CONCORD_E_NONPOS_DIAG, "constant column in X under STANDARDIZE");
  return CONCORD_OK;
}

int concord_tune_lambda(concord_state* st, const void* Sval_dev, int s_dtype, int lds, double lambda0,
                        int steps, double lr, double tol, int max_sweeps, double cg_tol,
                        double* rows_host) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!(lambda0 > 0.0) || steps < 1 || !(lr >= 0.0) || !rows_host || !(cg_tol > 0.0))
    return fail(CONCORD_E_ARG, "lambda0 > 0, steps >= 1, lr >= 0, cg_tol > 0, rows non-NULL");
  double log_lam = log(lambda0);
  for (int k = 0; k < steps; ++k) {
    const double lam = exp(log_lam);
    concord_result res;
    rc = concord_run(st, lam, tol, max_sweeps, CONCORD_STOP_KKT, 0.0, &res);
    if (rc < 0) return rc;
    double loss = 0.0;
    if ((rc = concord_heldout(st, Sval_dev, s_dtype, lds, &loss)) < 0) return rc;
    concord_adjoint_info info;
    if ((rc = concord_adjoint(st, nullptr, 0, 0, cg_tol, 10000, nullptr, 0, &info)) < 0) return rc;
    double* row = rows_host + 6 * (size_t)k;
    row[0] = lam;
    row[1] = loss;
    row[2] = info.dlambda;
    row[3] = res.sweeps;
    row[4] = info.iterations;
    row[5] = res.kkt;
    log_lam -= lr * lam * info.dlambda;
  }
  return CONCORD_OK;
}

int concord_get_omega_csr(concord_state* st, int32_t* rowptr, int32_t* col, double* val, int64_t cap,
                          int64_t* nnz_out) {
  int rc = check_state(st);
  if (rc) return rc;
  if (!rowptr || !nnz_out || cap < 0 || (cap > 0 && (!col || !val)))
    return fail(CONCORD_E_ARG, "rowptr and nnz non-NULL, cap >= 0, col / val non-NULL when cap > 0");
  const int p = st->p;
  const bool f64 = !is_mixed(st) || st->om64_current;
  const void* Om = f64 ? (const void*)st->Om64 : st->Om;
  if (!st->csr_rowptr) {
    CK(cudaMalloc(&st->csr_cnt, sizeof(int) * p));
    CK(cudaMalloc(&st->csr_rowptr, sizeof(int) * (p + 1)));
  }
  CK(launch_adj_count(Om, f64 ? 0 : 1, p, st->ld, st->csr_cnt, st->sms, st->stream));
  CK(launch_adj_scan(st->csr_cnt, p, st->csr_rowptr, st->stream));
  CK(cudaMemcpyAsync(st->h_flag, st->csr_rowptr + p, sizeof(int), cudaMemcpyDeviceToHost,
                     st->stream));
  CK(cudaStreamSynchronize(st->stream));
  const int nnz = *st->h_flag;
  *nnz_out = nnz;
  CK(cudaMemcpyAsync(rowptr, st->csr_rowptr, sizeof(int) * (p + 1), cudaMemcpyDefault, st->stream));
  if (nnz > cap) {
    CK(cudaStreamSynchronize(st->stream));
    return fail(CONCORD_E_ARG, "capacity %lld below the %d entries of Omega", (long long)cap, nnz);
  }
  if (nnz > st->csr_cap) {
    if (st->csr_col) cudaFree(st->csr_col);
    if (st->csr_row) cudaFree(st->csr_row);
    if (st->csr_val) cudaFree(st->csr_val);
    st->csr_col = st->csr_row = nullptr;
    st->csr_val = nullptr;
    st->csr_cap = 0;
    CK(cudaMalloc(&st->csr_col, sizeof(int) * (size_t)nnz));
    CK(cudaMalloc(&st->csr_row, sizeof(int) * (size_t)nnz));
    CK(cudaMalloc(&st->csr_val, sizeof(double) * (size_t)nnz));
    st->csr_cap = nnz;
  }
  CK(launch_adj_fill(Om, f64 ? 0 : 1, p, st->ld, st->csr_rowptr, st->csr_col, st->csr_row,
                     st->csr_val, st->sms, st->stream));
  CK(cudaMemcpyAsync(col, st->csr_col, sizeof(int) * (size_t)nnz, cudaMemcpyDefault, st->stream));
  CK(cudaMemcpyAsync(val, st->csr_val, sizeof(double) * (size_t)nnz, cudaMemcpyDefault,
                     st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CK(cudaGetLastError());
  return CONCORD_OK;
}

}  // extern "C"
