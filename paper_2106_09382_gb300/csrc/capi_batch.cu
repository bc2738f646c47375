// Host side of the batched entry points (concord_batch_*) of the C ABI in
// include/concord.h: many independent CONCORD problems (uneven p and n) in
// one persistent launch of the sweep kernel per wave of co-resident
// problems, each problem walking a warm-started lambda path.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "concord.h"
#include "kernels.h"
#include "prep_stats.h"

using namespace concord;

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define BCK(expr)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      if (e_ == cudaErrorMemoryAllocation)                                               \
        return bfail(CONCORD_E_NOMEM, "%s: %s", #expr, cudaGetErrorString(e_));          \
      if (e_ == cudaErrorCooperativeLaunchTooLarge)                                      \
        return bfail(CONCORD_E_OCCUPANCY, "%s: %s", #expr, cudaGetErrorString(e_));      \
      return bfail(CONCORD_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
    }                                                                                    \
  } while (0)

int rup(int v, int m) { return (v + m - 1) / m * m; }

constexpr int kBatchWarps = kSweepThreads / 32;  // warps per CTA, all owning rows
constexpr int kRowsChoices[] = {32, 16, 8, 4, 2};

// One problem's device arrays (T = float for CONCORD_MIXED, double for FP64).
struct Prob {
  int p = 0, P = 0, pe = 0, ld = 0;
  void *S = nullptr, *W = nullptr, *Om = nullptr, *sdiagT = nullptr, *sd1 = nullptr,
       *sd2 = nullptr;
  double *sdiag64 = nullptr, *omdiag64 = nullptr, *partials = nullptr;
  // MIXED: FP64 copies for the polish of a lambda whose FP32 sweeps stall
  double *S64 = nullptr, *W64 = nullptr, *Om64 = nullptr, *sd1_64 = nullptr, *sd2_64 = nullptr;
  unsigned long long* mbox = nullptr;
  unsigned* barrier = nullptr;
  bool have_S = false;
};

// One problem's share of a launch: it walks lambdas[k0 .. k0 + nk).
struct Item {
  int b, k0, nk, stall_break, n_sweeps;
};

}  // namespace

struct concord_batch {
  int device = -1, sms = 0, precision = 0, n_cap = 0, pmax = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  std::vector<Prob> probs;
  double timeout_s = 2.0;
  int rows_per_warp = 0;  // 0: autotune on the first path call
  bool polish = true;     // MIXED: FP64 polish of a lambda whose FP32 sweeps stall
  int last_ctas = 0, last_waves = 0;
  // data staging for concord_batch_gram (one problem at a time)
  double *Xg = nullptr, *mean = nullptr, *inv = nullptr, *part = nullptr;
  float *zt_hi = nullptr, *zt_lo = nullptr;
  void* Z = nullptr;
  int* flag = nullptr;
  int* h_flag = nullptr;
  // launch scratch
  int* abort_info = nullptr;
  double* lam_dev = nullptr;
  int lam_cap = 0;
  double* res_dev = nullptr;
  size_t res_cap = 0;
  void* probs_dev = nullptr;
  size_t probs_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.f;
};

namespace {

bool is_mixed(const concord_batch* bt) { return bt->precision == CONCORD_MIXED; }
size_t esz(const concord_batch* bt) { return is_mixed(bt) ? 4 : 8; }

void free_prob(Prob& q) {
  void* d[] = {q.S,        q.W,      q.Om,     q.sdiagT, q.sd1,    q.sd2,  q.sdiag64,
               q.omdiag64, q.partials, q.mbox, q.barrier, q.S64, q.W64, q.Om64,
               q.sd1_64,   q.sd2_64};
  for (void* x : d)
    if (x) cudaFree(x);
  q = Prob();
}

void free_all(concord_batch* bt) {
  for (auto& q : bt->probs) free_prob(q);
  void* d[] = {bt->Xg, bt->mean, bt->inv, bt->part, bt->zt_hi, bt->zt_lo, bt->Z, bt->flag, bt->abort_info,
               bt->lam_dev, bt->res_dev, bt->probs_dev};
  for (void* x : d)
    if (x) cudaFree(x);
  if (bt->h_flag) cudaFreeHost(bt->h_flag);
  if (bt->ev0) cudaEventDestroy(bt->ev0);
  if (bt->ev1) cudaEventDestroy(bt->ev1);
  if (bt->own_stream) cudaStreamDestroy(bt->own_stream);
}

int check_b(concord_batch* bt, int b) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (b < 0 || b >= (int)bt->probs.size())
    return bfail(CONCORD_E_ARG, "problem index %d out of range (0..%d)", b,
                 (int)bt->probs.size() - 1);
  return CONCORD_OK;
}

// Omega_b = I, W_b = S_b, diagonals and walk vectors from S_b.
int reset_prob(concord_batch* bt, Prob& q) {
  const int f32 = is_mixed(bt) ? 1 : 0;
  cudaStream_t s = bt->stream;
  BCK(cudaMemsetAsync(bt->flag, 0, sizeof(int), s));
  if (f32) {  // the FP64 diagonal from the FP64 copy of S, as a single state keeps it
    BCK(launch_extract_diag(q.S64, 0, q.ld, q.p, q.sdiag64, q.sdiagT, 1, bt->flag, s));
    BCK(launch_fill_f64(q.omdiag64, 1.0, q.p, s));
  } else {
    BCK(launch_extract_diag(q.S, 0, q.ld, q.p, q.sdiag64, nullptr, 0, bt->flag, s));
    BCK(cudaMemcpyAsync(q.sdiagT, q.sdiag64, sizeof(double) * q.p, cudaMemcpyDeviceToDevice, s));
  }
  BCK(launch_subdiag(q.S, f32, q.ld, q.p, q.P, q.sd1, q.sd2, s));
  if (f32) BCK(launch_subdiag(q.S64, 0, q.ld, q.p, q.P, q.sd1_64, q.sd2_64, s));
  BCK(launch_set_identity(q.Om, f32, q.p, q.ld, s));
  BCK(cudaMemcpyAsync(q.W, q.S, esz(bt) * (size_t)q.p * q.ld, cudaMemcpyDeviceToDevice, s));
  BCK(cudaMemcpyAsync(bt->h_flag, bt->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  if (*bt->h_flag & 2) return bfail(CONCORD_E_NONFINITE, "S has a non-finite diagonal entry");
  if (*bt->h_flag & 1) return bfail(CONCORD_E_NONPOS_DIAG, "S has a non-positive diagonal entry");
  q.have_S = true;
  return CONCORD_OK;
}

// CTAs a problem of dimension p takes at `rows` rows per warp.
int ctas_for(int p, int rows) {
  const int per_cta = kBatchWarps * rows;
  return (p + per_cta - 1) / per_cta;
}

// One launch per wave of co-resident items.  T = float: the FP32 arrays of
// a MIXED batch; T = double: the arrays of an FP64 batch, or the FP64 copies
// of a MIXED batch (its polish).  Result rows land at [b][k] of the batch's
// n_problems x n_lambda table, copied back into res_host.
template <typename T>
int run_waves(concord_batch* bt, int rows, const std::vector<Item>& items,
              const double* lambdas_host, int n_lambda, double tol, int max_sweeps, int stall_stop,
              float* support_dev, std::vector<double>* res_host) {
  cudaStream_t s = bt->stream;
  const int B = (int)bt->probs.size();
  const int nI = (int)items.size();
  const bool copies = sizeof(T) == 8 && is_mixed(bt);
  int occ = 0;
  BCK(sweep_occupancy(sizeof(T) == 4, kSweepThreads, &occ));
  if (occ < 1) return bfail(CONCORD_E_OCCUPANCY, "sweep kernel cannot be resident");
  const int capacity = bt->sms * occ;
  for (const auto& it : items)
    if (ctas_for(bt->probs[it.b].p, rows) > capacity)
      return bfail(CONCORD_E_ARG, "p=%d needs more than %d CTAs at %d rows per warp",
                   bt->probs[it.b].p, capacity, rows);
  // device copies of the lambdas, the result rows and the problem table
  if (n_lambda > bt->lam_cap) {
    if (bt->lam_dev) cudaFree(bt->lam_dev);
    bt->lam_dev = nullptr;
    BCK(cudaMalloc(&bt->lam_dev, sizeof(double) * n_lambda));
    bt->lam_cap = n_lambda;
  }
  BCK(cudaMemcpyAsync(bt->lam_dev, lambdas_host, sizeof(double) * n_lambda,
                      cudaMemcpyHostToDevice, s));
  const size_t nres = (size_t)B * n_lambda * kRes;
  if (nres > bt->res_cap) {
    if (bt->res_dev) cudaFree(bt->res_dev);
    bt->res_dev = nullptr;
    BCK(cudaMalloc(&bt->res_dev, sizeof(double) * nres));
    bt->res_cap = nres;
  }
  BCK(cudaMemsetAsync(bt->res_dev, 0, sizeof(double) * nres, s));
  if ((size_t)nI * sizeof(BatchProblem<T>) > bt->probs_cap) {
    if (bt->probs_dev) cudaFree(bt->probs_dev);
    bt->probs_dev = nullptr;
    BCK(cudaMalloc(&bt->probs_dev, (size_t)nI * sizeof(BatchProblem<T>)));
    bt->probs_cap = (size_t)nI * sizeof(BatchProblem<T>);
  }
  // greedy waves of consecutive items whose CTAs fit co-resident
  std::vector<std::pair<int, int>> waves;
  {
    int i0 = 0, used = 0;
    for (int i = 0; i < nI; ++i) {
      const int c = ctas_for(bt->probs[items[i].b].p, rows);
      if (used + c > capacity && i > i0) {
        waves.push_back({i0, i});
        i0 = i;
        used = 0;
      }
      used += c;
    }
    if (i0 < nI) waves.push_back({i0, nI});
  }
  std::vector<BatchProblem<T>> table(nI);
  for (const auto& w : waves) {
    int cta0 = 0;
    for (int i = w.first; i < w.second; ++i) {
      const Item& it = items[i];
      Prob& q = bt->probs[it.b];
      BatchProblem<T>& e = table[i];
      memset(&e, 0, sizeof e);
      e.p = q.p;
      e.P = q.P;
      e.ld = q.ld;
      e.cta0 = cta0;
      e.ctas = ctas_for(q.p, rows);
      cta0 += e.ctas;
      e.W = (T*)(copies ? (void*)q.W64 : q.W);
      e.Om = (T*)(copies ? (void*)q.Om64 : q.Om);
      e.S = (const T*)(copies ? (void*)q.S64 : q.S);
      e.sdiag = (const T*)(copies ? (void*)q.sdiag64 : q.sdiagT);
      e.sd1 = (const T*)(copies ? (void*)q.sd1_64 : q.sd1);
      e.sd2 = (const T*)(copies ? (void*)q.sd2_64 : q.sd2);
      e.sdiag64 = q.sdiag64;
      e.omdiag64 = sizeof(T) == 4 ? q.omdiag64 : nullptr;
      e.mbox = q.mbox;
      e.barrier = q.barrier;
      e.partials = q.partials;
      e.result = bt->res_dev + ((size_t)it.b * n_lambda + it.k0) * kRes;
      e.cnt = support_dev ? support_dev + (size_t)it.k0 * q.p * q.p : nullptr;
      e.k0 = it.k0;
      e.nk = it.nk;
      e.stall_break = it.stall_break;
      e.n_sweeps = it.n_sweeps;
      // fresh mailboxes: this launch's step tags start at 1
      BCK(cudaMemsetAsync(q.mbox, 0, sizeof(unsigned long long) * 2 * (size_t)kDepth * q.pe, s));
      BCK(cudaMemsetAsync(q.barrier, 0, sizeof(unsigned), s));
    }
  }
  BCK(cudaMemcpyAsync(bt->probs_dev, table.data(), (size_t)nI * sizeof(BatchProblem<T>),
                      cudaMemcpyHostToDevice, s));
  BCK(cudaMemsetAsync(bt->abort_info, 0, 3 * sizeof(int), s));
  BCK(cudaEventRecord(bt->ev0, s));
  int total_ctas = 0;
  for (const auto& w : waves) {
    SweepArgs<T> a;
    memset(&a, 0, sizeof a);
    const BatchProblem<T>& first = table[w.first];
    a.p = first.p;
    a.P = first.P;
    a.ld = first.ld;
    a.rows_per_warp = rows;
    a.row_warps = kBatchWarps;
    a.depth = kDepth;
    a.wait.abort = bt->abort_info;
    a.wait.info = bt->abort_info + 1;
    a.wait.timeout_ns = (uint64_t)(bt->timeout_s * 1e9);
    a.lambda = lambdas_host[0];
    a.tol = tol;
    a.delta_tol = 1e-5;
    a.stop_rule = CONCORD_STOP_KKT;
    a.n_sweeps = max_sweeps;
    a.stall_stop = stall_stop;
    a.tag_base = 1;
    a.fault_vertex = -1;
    a.fault_step = -1;
    a.probs = (const BatchProblem<T>*)bt->probs_dev + w.first;
    a.n_probs = w.second - w.first;
    a.lambdas = bt->lam_dev;
    a.n_lambda = n_lambda;
    int grid = 0;
    for (int i = w.first; i < w.second; ++i) grid += table[i].ctas;
    total_ctas = std::max(total_ctas, grid);
    BCK(launch_sweep_batch(a, grid, kSweepThreads, s));
  }
  BCK(cudaEventRecord(bt->ev1, s));
  res_host->assign(nres, 0.0);
  BCK(cudaMemcpyAsync(res_host->data(), bt->res_dev, sizeof(double) * nres,
                      cudaMemcpyDeviceToHost, s));
  int h_abort[3] = {0, 0, 0};
  BCK(cudaMemcpyAsync(h_abort, bt->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  BCK(cudaGetLastError());
  float ms = 0.f;
  BCK(cudaEventElapsedTime(&ms, bt->ev0, bt->ev1));
  bt->last_ms = ms;
  bt->last_ctas = std::max(bt->last_ctas, total_ctas);
  bt->last_waves = std::max(bt->last_waves, (int)waves.size());
  if (h_abort[0] != 0)
    return bfail(CONCORD_E_TIMEOUT, "batched sweep: a device wait ran out (where %d, step %d)",
                 h_abort[1], h_abort[2]);
  return CONCORD_OK;
}

std::vector<Item> all_items(const concord_batch* bt, int n_lambda, int stall_break) {
  std::vector<Item> items;
  for (int b = 0; b < (int)bt->probs.size(); ++b) items.push_back({b, 0, n_lambda, stall_break, 0});
  return items;
}

int run_any(concord_batch* bt, int rows, const double* lambdas, int n_lambda, double tol,
            int max_sweeps, float* support_dev, std::vector<double>* res) {
  const auto items = all_items(bt, n_lambda, 0);
  bt->last_ctas = bt->last_waves = 0;
  return is_mixed(bt) ? run_waves<float>(bt, rows, items, lambdas, n_lambda, tol, max_sweeps, 1,
                                         support_dev, res)
                      : run_waves<double>(bt, rows, items, lambdas, n_lambda, tol, max_sweeps, 0,
                                          support_dev, res);
}

// MIXED polish of problem b: FP64 copies from the FP32 iterate (W rebuilt in
// FP64 from Omega and S64) / the FP32 working set back from them.
int promote(concord_batch* bt, Prob& q) {
  cudaStream_t s = bt->stream;
  BCK(launch_convert(q.Om, 1, q.ld, q.Om64, 0, q.ld, q.p, q.p, s));
  BCK(cudaMemcpy2DAsync(q.Om64, (size_t)(q.ld + 1) * sizeof(double), q.omdiag64, sizeof(double),
                        sizeof(double), q.p, cudaMemcpyDeviceToDevice, s));
  BCK(launch_refresh_w(q.Om64, q.S64, q.W64, q.p, q.ld, bt->sms, s));
  return CONCORD_OK;
}
int demote(concord_batch* bt, Prob& q) {
  cudaStream_t s = bt->stream;
  BCK(launch_convert(q.Om64, 0, q.ld, q.Om, 1, q.ld, q.p, q.p, s));
  BCK(launch_convert(q.W64, 0, q.ld, q.W, 1, q.ld, q.p, q.p, s));
  BCK(cudaMemcpy2DAsync(q.omdiag64, sizeof(double), q.Om64, (size_t)(q.ld + 1) * sizeof(double),
                        sizeof(double), q.p, cudaMemcpyDeviceToDevice, s));
  return CONCORD_OK;
}

// The MIXED path with polish: the FP32 launches walk every problem's path
// until a lambda's sweeps stall (the problem's walk ends there); those
// lambdas are polished in FP64 (one launch for all of them), their support
// counted from the FP64 iterate, and the walks resume after them.
int mixed_path(concord_batch* bt, int rows, const double* lambdas, int n_lambda, double tol,
               int max_sweeps, float* support_dev, std::vector<double>* R,
               std::vector<int>* sweeps32) {
  const int B = (int)bt->probs.size();
  R->assign((size_t)B * n_lambda * kRes, 0.0);
  sweeps32->assign((size_t)B * n_lambda, 0);
  std::vector<int> next(B, 0);
  std::vector<double> res;
  bt->last_ctas = bt->last_waves = 0;
  float total_ms = 0.f;
  for (;;) {
    std::vector<Item> items;
    for (int b = 0; b < B; ++b)
      if (next[b] < n_lambda) items.push_back({b, next[b], n_lambda - next[b], 1, 0});
    if (items.empty()) break;
    int rc = run_waves<float>(bt, rows, items, lambdas, n_lambda, tol, max_sweeps, 1, support_dev,
                              &res);
    if (rc != CONCORD_OK) return rc;
    total_ms += bt->last_ms;
    std::vector<Item> pol;
    for (const Item& it : items) {
      int k = it.k0;
      for (; k < n_lambda; ++k) {
        const double* x = res.data() + ((size_t)it.b * n_lambda + k) * kRes;
        const size_t o = ((size_t)it.b * n_lambda + k) * kRes;
        for (int q = 0; q < kRes; ++q) (*R)[o + q] = x[q];
        (*sweeps32)[(size_t)it.b * n_lambda + k] = (int)x[kResSweeps];
        const int code = (int)x[kResStatus];
        if (code == 4) break;              // stalled: polish it
        if (code == 2 || code == 3) {      // non-finite / aborted: the walk ended
          k = n_lambda;
          break;
        }
      }
      if (k < n_lambda) {
        const int done = (*sweeps32)[(size_t)it.b * n_lambda + k];
        pol.push_back({it.b, k, 1, 0, max_sweeps > done ? max_sweeps - done : 1});
        next[it.b] = k;
      } else {
        next[it.b] = n_lambda;
      }
    }
    if (pol.empty()) break;
    for (const Item& it : pol)
      if ((rc = promote(bt, bt->probs[it.b])) != CONCORD_OK) return rc;
    rc = run_waves<double>(bt, rows, pol, lambdas, n_lambda, tol, max_sweeps, 0, nullptr, &res);
    if (rc != CONCORD_OK) return rc;
    total_ms += bt->last_ms;
    for (const Item& it : pol) {
      Prob& q = bt->probs[it.b];
      if ((rc = demote(bt, q)) != CONCORD_OK) return rc;
      if (support_dev)
        BCK(launch_support_add(q.Om64, 0, q.ld, q.p, support_dev + (size_t)it.k0 * q.p * q.p,
                               bt->stream));
      const size_t o = ((size_t)it.b * n_lambda + it.k0) * kRes;
      const double* x = res.data() + o;
      const double s32 = (*R)[o + kResSweeps];
      for (int q2 = 0; q2 < kRes; ++q2) (*R)[o + q2] = x[q2];
      (*R)[o + kResSweeps] = s32 + x[kResSweeps];
      next[it.b] = it.k0 + 1;
    }
  }
  BCK(cudaStreamSynchronize(bt->stream));
  bt->last_ms = total_ms;
  return CONCORD_OK;
}

void fill_results(const std::vector<double>& r, const std::vector<int>* sweeps32, int B,
                  int n_lambda, const double* lambdas, concord_result* out) {
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < n_lambda; ++k) {
      const double* x = r.data() + ((size_t)b * n_lambda + k) * kRes;
      concord_result& o = out[(size_t)b * n_lambda + k];
      memset(&o, 0, sizeof o);
      const int code = (int)x[kResStatus];
      o.status = code == 0 ? CONCORD_OK
                 : code == 2 ? CONCORD_E_NONFINITE
                 : code == 3 ? CONCORD_E_TIMEOUT
                             : CONCORD_NOT_CONVERGED;
      o.sweeps = (int)x[kResSweeps];
      o.first_delta_sweep = (int)x[kResFirstDelta];
      o.objective = x[kResObj];
      o.kkt = x[kResKkt];
      o.delta = x[kResDelta];
      o.lambda = lambdas[k];
      o.active_pairs = (long long)(x[kResActive] + 0.5);
      o.timeout_vertex = -1;
      o.timeout_step = -1;
      o.dense_sweeps = o.sweeps;
      if (sweeps32) o.sweeps_fp32 = (*sweeps32)[(size_t)b * n_lambda + k];
    }
}

}  // namespace

int concord_batch_create(concord_batch** out, int n_problems, const int* p, int precision,
                         int n_cap, int device) {
  if (!out) return bfail(CONCORD_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_problems < 1 || !p || n_cap < 0 ||
      (precision != CONCORD_FP64 && precision != CONCORD_MIXED))
    return bfail(CONCORD_E_ARG, "n_problems >= 1, p non-NULL, n_cap >= 0, precision FP64/MIXED");
  for (int b = 0; b < n_problems; ++b)
    if (p[b] < 2) return bfail(CONCORD_E_ARG, "p[%d] = %d (must be >= 2)", b, p[b]);
  if (device < 0 && cudaGetDevice(&device) != cudaSuccess)
    return bfail(CONCORD_E_CUDA, "no CUDA device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
    return bfail(CONCORD_E_CUDA, "cannot query device %d", device);
  if (prop.major != 10 || prop.minor != 3)
    return bfail(CONCORD_E_CUDA, "device %d is sm_%d%d; this library is built for sm_103",
                 device, prop.major, prop.minor);
  BCK(cudaSetDevice(device));
  concord_batch* bt = new concord_batch;
  bt->device = device;
  bt->sms = prop.multiProcessorCount;
  bt->precision = precision;
  bt->n_cap = n_cap;
  bt->probs.resize(n_problems);
  int rc = CONCORD_OK;
  const size_t e = esz(bt);
#define BALLOC(ptr, bytes)                                                        \
  do {                                                                            \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                     \
      rc = bfail(CONCORD_E_NOMEM, "cudaMalloc of %zu bytes failed", (size_t)(bytes)); \
      goto fail_out;                                                              \
    }                                                                             \
  } while (0)
  if (cudaStreamCreateWithFlags(&bt->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    rc = bfail(CONCORD_E_CUDA, "cudaStreamCreate failed");
    goto fail_out;
  }
  bt->stream = bt->own_stream;
  for (int b = 0; b < n_problems; ++b) {
    Prob& q = bt->probs[b];
    q.p = p[b];
    q.pe = p[b] + (p[b] & 1);
    q.P = q.pe - 1;
    q.ld = rup(p[b], kTile);
    bt->pmax = std::max(bt->pmax, q.p);
    const size_t mat = e * (size_t)q.p * q.ld;
    BALLOC(q.S, mat);
    BALLOC(q.W, mat);
    BALLOC(q.Om, mat);
    BALLOC(q.sdiagT, e * q.p);
    BALLOC(q.sd1, e * (q.P + 1));
    BALLOC(q.sd2, e * (q.P + 1));
    BALLOC(q.sdiag64, sizeof(double) * q.p);
    BALLOC(q.omdiag64, sizeof(double) * q.p);
    BALLOC(q.partials, sizeof(double) * kParts * (size_t)ctas_for(q.p, 2));
    BALLOC(q.mbox, sizeof(unsigned long long) * 2 * (size_t)kDepth * q.pe);
    BALLOC(q.barrier, sizeof(unsigned));
    if (e == 4) {
      const size_t mat64 = sizeof(double) * (size_t)q.p * q.ld;
      BALLOC(q.S64, mat64);
      BALLOC(q.W64, mat64);
      BALLOC(q.Om64, mat64);
      BALLOC(q.sd1_64, sizeof(double) * (q.P + 1));
      BALLOC(q.sd2_64, sizeof(double) * (q.P + 1));
      cudaMemsetAsync(q.S64, 0, mat64, bt->stream);
      launch_set_identity(q.S64, 0, q.p, q.ld, bt->stream);
    }
    cudaMemsetAsync(q.S, 0, mat, bt->stream);
    launch_set_identity(q.S, e == 4 ? 1 : 0, q.p, q.ld, bt->stream);
  }
  BALLOC(bt->flag, sizeof(int));
  BALLOC(bt->abort_info, 3 * sizeof(int));
  if (n_cap > 0) {
    const int n_pad = rup(n_cap, 64), p_pad = rup(bt->pmax, 128);
    BALLOC(bt->Xg, sizeof(double) * (size_t)n_cap * bt->pmax);
    BALLOC(bt->mean, sizeof(double) * bt->pmax);
    BALLOC(bt->inv, sizeof(double) * bt->pmax);
    BALLOC(bt->part, sizeof(double) * (size_t)col_stats_chunks(n_cap) * bt->pmax);
    if (is_mixed(bt)) {
      BALLOC(bt->zt_hi, sizeof(float) * (size_t)n_pad * p_pad);
      BALLOC(bt->zt_lo, sizeof(float) * (size_t)n_pad * p_pad);
    } else {
      BALLOC(bt->Z, sizeof(double) * (size_t)n_cap * rup(bt->pmax, kTile));
    }
  }
#undef BALLOC
  if (cudaMallocHost((void**)&bt->h_flag, sizeof(int)) != cudaSuccess ||
      cudaEventCreate(&bt->ev0) != cudaSuccess || cudaEventCreate(&bt->ev1) != cudaSuccess) {
    rc = bfail(CONCORD_E_CUDA, "host allocation or event creation failed");
    goto fail_out;
  }
  if (cudaStreamSynchronize(bt->stream) != cudaSuccess) {
    rc = bfail(CONCORD_E_CUDA, "initialisation failed");
    goto fail_out;
  }
  for (auto& q : bt->probs)
    if ((rc = reset_prob(bt, q)) != CONCORD_OK) goto fail_out;
  for (auto& q : bt->probs) q.have_S = false;
  *out = bt;
  return CONCORD_OK;
fail_out:
  free_all(bt);
  delete bt;
  return rc;
}

int concord_batch_destroy(concord_batch* bt) {
  if (!bt) return CONCORD_OK;
  cudaSetDevice(bt->device);
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  free_all(bt);
  delete bt;
  return CONCORD_OK;
}

int concord_batch_set_stream(concord_batch* bt, void* stream) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  bt->stream = stream ? (cudaStream_t)stream : bt->own_stream;
  return CONCORD_OK;
}

int concord_batch_set_timeout(concord_batch* bt, double seconds) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (!(seconds > 0.0) || seconds > 3600.0) return bfail(CONCORD_E_ARG, "timeout in (0, 3600] s");
  bt->timeout_s = seconds;
  return CONCORD_OK;
}

int concord_batch_set_polish(concord_batch* bt, int on) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (on != 0 && on != 1) return bfail(CONCORD_E_ARG, "on must be 0 or 1");
  bt->polish = on == 1;
  return CONCORD_OK;
}

int concord_batch_set_rows_per_warp(concord_batch* bt, int rows) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (rows != 0 && rows != 2 && rows != 4 && rows != 8 && rows != 16 && rows != 32)
    return bfail(CONCORD_E_ARG, "rows per warp must be 0 (autotune), 2, 4, 8, 16 or 32");
  bt->rows_per_warp = rows;
  return CONCORD_OK;
}

int concord_batch_info(concord_batch* bt, int* rows_per_warp, int* ctas, int* waves,
                       double* seconds) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (rows_per_warp) *rows_per_warp = bt->rows_per_warp;
  if (ctas) *ctas = bt->last_ctas;
  if (waves) *waves = bt->last_waves;
  if (seconds) *seconds = bt->last_ms * 1e-3;
  return CONCORD_OK;
}

int concord_batch_set_S(concord_batch* bt, int b, const void* S_dev, int s_dtype, int lds) {
  int rc = check_b(bt, b);
  if (rc) return rc;
  Prob& q = bt->probs[b];
  if (!S_dev || (s_dtype != CONCORD_F64 && s_dtype != CONCORD_F32) || lds < q.p)
    return bfail(CONCORD_E_ARG, "S_dev non-NULL, dtype F64/F32, lds >= p required");
  BCK(cudaSetDevice(bt->device));
  const int f32 = s_dtype == CONCORD_F32;
  BCK(cudaMemsetAsync(bt->flag, 0, sizeof(int), bt->stream));
  BCK(launch_check_symmetric(S_dev, f32, q.p, lds, bt->flag, bt->stream));
  BCK(cudaMemcpyAsync(bt->h_flag, bt->flag, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
  BCK(cudaStreamSynchronize(bt->stream));
  if (*bt->h_flag & 2) return bfail(CONCORD_E_NONFINITE, "S has a non-finite entry");
  if (*bt->h_flag & 1) return bfail(CONCORD_E_ARG, "S is not symmetric");
  BCK(launch_convert(S_dev, f32, lds, q.S, is_mixed(bt) ? 1 : 0, q.ld, q.p, q.p, bt->stream));
  if (is_mixed(bt))
    BCK(launch_convert(S_dev, f32, lds, q.S64, 0, q.ld, q.p, q.p, bt->stream));
  return reset_prob(bt, q);
}

int concord_batch_gram(concord_batch* bt, int b, const void* X_dev, int x_dtype, int n, int ldx,
                       const int* rows_dev, int n_rows, int prep) {
  int rc = check_b(bt, b);
  if (rc) return rc;
  Prob& q = bt->probs[b];
  const int nr = rows_dev ? n_rows : n;
  if (!X_dev || n < 1 || ldx < q.p || (x_dtype != CONCORD_F64 && x_dtype != CONCORD_F32) ||
      prep < 0 || prep > 2 || nr < 1)
    return bfail(CONCORD_E_ARG, "bad argument to concord_batch_gram");
  if (nr > bt->n_cap)
    return bfail(CONCORD_E_ARG, "%d data rows exceed the batch's n_cap (%d)", nr, bt->n_cap);
  BCK(cudaSetDevice(bt->device));
  cudaStream_t s = bt->stream;
  const int x_f32 = x_dtype == CONCORD_F32;
  const int p = q.p;
  // the problem's rows, dense FP64 (nr x p)
  if (rows_dev) {
    BCK(launch_gather_rows(X_dev, x_f32, ldx, rows_dev, nr, p, bt->Xg, s));
  } else {
    BCK(launch_convert(X_dev, x_f32, ldx, bt->Xg, 0, p, nr, p, s));
  }
  BCK(cudaMemsetAsync(bt->flag, 0, sizeof(int), s));
  BCK(launch_col_stats_chunked(bt->Xg, 0, nr, p, p, prep, bt->mean, bt->inv, bt->flag, bt->part,
                               s));
  if (is_mixed(bt)) {
    const int n_pad = rup(nr, 32), p_pad = rup(p, 128);
    BCK(launch_split_tf32(bt->Xg, 0, nr, p, p, bt->mean, bt->inv, bt->zt_hi, bt->zt_lo, n_pad,
                          p_pad, s));
    cudaError_t e = launch_gram_tf32x3(bt->zt_hi, bt->zt_lo, n_pad, p_pad, p, (float*)q.S, q.ld,
                                       1.0f / nr, bt->flag, s);
    if (e == cudaErrorNotSupported) return bfail(CONCORD_E_CUDA, "tensor-core Gram unavailable");
    BCK(e);
    BCK(launch_convert(q.S, 1, q.ld, q.S64, 0, q.ld, p, p, s));
  } else {
    const int ldz = rup(p, kTile);
    BCK(launch_apply_prep(bt->Xg, 0, nr, p, p, bt->mean, bt->inv, bt->Z, 0, ldz, s));
    BCK(launch_syrk_f64((const double*)bt->Z, nr, p, ldz, (double*)q.S, q.ld, 1.0 / nr, s));
  }
  BCK(cudaMemcpyAsync(bt->h_flag, bt->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  const int bad = *bt->h_flag;
  if (bad & 4) return bfail(CONCORD_E_TIMEOUT, "tensor-core Gram: a device-side wait ran out");
  if (bad & 2) return bfail(CONCORD_E_NONFINITE, "X has a non-finite entry");
  if (bad & 1) return bfail(CONCORD_E_NONPOS_DIAG, "X has a constant column");
  return reset_prob(bt, q);
}

int concord_batch_reset(concord_batch* bt, int b) {
  int rc = check_b(bt, b);
  if (rc) return rc;
  if (!bt->probs[b].have_S) return bfail(CONCORD_E_ARG, "problem %d has no S yet", b);
  BCK(cudaSetDevice(bt->device));
  return reset_prob(bt, bt->probs[b]);
}

int concord_batch_autotune(concord_batch* bt, double lambda, int sweeps, double* ms_per_choice) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (!(lambda >= 0.0) || sweeps < 1) return bfail(CONCORD_E_ARG, "lambda >= 0, sweeps >= 1");
  for (auto& q : bt->probs)
    if (!q.have_S) return bfail(CONCORD_E_ARG, "every problem needs S before autotuning");
  BCK(cudaSetDevice(bt->device));
  int best = 0;
  float best_ms = 0.f;
  int i = 0;
  for (int rows : kRowsChoices) {
    std::vector<double> res;
    int rc = run_any(bt, rows, &lambda, 1, -1.0, sweeps, nullptr, &res);
    float ms = rc == CONCORD_OK ? bt->last_ms : -1.f;
    if (ms_per_choice) ms_per_choice[i] = ms;
    ++i;
    if (rc == CONCORD_E_TIMEOUT || rc == CONCORD_E_CUDA) return rc;
    if (ms > 0.f && (best == 0 || ms < best_ms)) {
      best = rows;
      best_ms = ms;
    }
    for (auto& q : bt->probs)
      if ((rc = reset_prob(bt, q)) != CONCORD_OK) return rc;
  }
  if (best == 0) return bfail(CONCORD_E_OCCUPANCY, "no rows-per-warp choice could launch");
  bt->rows_per_warp = best;
  return CONCORD_OK;
}

int concord_batch_path(concord_batch* bt, const double* lambdas, int n_lambda, double tol,
                       int max_sweeps, concord_result* results, float* support_dev) {
  if (!bt) return bfail(CONCORD_E_ARG, "batch is NULL");
  if (!lambdas || n_lambda < 1 || !(tol > 0.0) || max_sweeps < 1)
    return bfail(CONCORD_E_ARG, "lambdas non-NULL, n_lambda >= 1, tol > 0, max_sweeps >= 1");
  for (int k = 0; k < n_lambda; ++k)
    if (!(lambdas[k] >= 0.0)) return bfail(CONCORD_E_ARG, "lambda[%d] must be >= 0", k);
  for (size_t b = 0; b < bt->probs.size(); ++b) {
    if (!bt->probs[b].have_S) return bfail(CONCORD_E_ARG, "problem %d has no S yet", (int)b);
    if (support_dev && bt->probs[b].p != bt->probs[0].p)
      return bfail(CONCORD_E_ARG, "support counts need every problem to have the same p");
  }
  if ((long long)n_lambda * max_sweeps * (bt->pmax + 1) >= (1ll << 31))
    return bfail(CONCORD_E_ARG, "n_lambda x max_sweeps x p must stay below 2^31");
  BCK(cudaSetDevice(bt->device));
  int rc;
  if (bt->rows_per_warp == 0) {
    // autotune on a short run at the path's middle lambda, then start over
    std::vector<double> ms(5);
    if ((rc = concord_batch_autotune(bt, lambdas[n_lambda / 2], 2, ms.data())) != CONCORD_OK)
      return rc;
  }
  std::vector<double> res;
  if (is_mixed(bt) && bt->polish) {
    std::vector<int> s32;
    rc = mixed_path(bt, bt->rows_per_warp, lambdas, n_lambda, tol, max_sweeps, support_dev, &res,
                    &s32);
    if (rc != CONCORD_OK) return rc;
    if (results) fill_results(res, &s32, (int)bt->probs.size(), n_lambda, lambdas, results);
    return CONCORD_OK;
  }
  rc = run_any(bt, bt->rows_per_warp, lambdas, n_lambda, tol, max_sweeps, support_dev, &res);
  if (rc != CONCORD_OK) return rc;
  if (results) {
    std::vector<int> s32;
    if (is_mixed(bt))
      for (size_t q = 0; q < res.size() / kRes; ++q) s32.push_back((int)res[q * kRes + kResSweeps]);
    fill_results(res, is_mixed(bt) ? &s32 : nullptr, (int)bt->probs.size(), n_lambda, lambdas,
                 results);
  }
  return CONCORD_OK;
}

int concord_batch_get_omega(concord_batch* bt, int b, void* out_dev, int dtype, int ldo) {
  int rc = check_b(bt, b);
  if (rc) return rc;
  Prob& q = bt->probs[b];
  if (!out_dev || (dtype != CONCORD_F64 && dtype != CONCORD_F32) || ldo < q.p)
    return bfail(CONCORD_E_ARG, "out non-NULL, dtype F64/F32, ldo >= p required");
  BCK(cudaSetDevice(bt->device));
  const int f32 = is_mixed(bt) ? 1 : 0;
  BCK(launch_convert(q.Om, f32, q.ld, out_dev, dtype == CONCORD_F32 ? 1 : 0, ldo, q.p, q.p,
                     bt->stream));
  if (f32 && dtype == CONCORD_F64)  // the FP64 diagonal of the mixed iterate
    BCK(cudaMemcpy2DAsync(out_dev, (size_t)(ldo + 1) * sizeof(double), q.omdiag64, sizeof(double),
                          sizeof(double), q.p, cudaMemcpyDeviceToDevice, bt->stream));
  BCK(cudaStreamSynchronize(bt->stream));
  return CONCORD_OK;
}
