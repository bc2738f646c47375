// Host side of the joint two-population entry points (concord_joint_*) of the
// C ABI declared in include/concord.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "concord.h"
#include "joint.h"
#include "kernels.h"

using namespace concord;

namespace {

int jfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define JCK(expr)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      if (e_ == cudaErrorMemoryAllocation)                                               \
        return jfail(CONCORD_E_NOMEM, "%s: %s", #expr, cudaGetErrorString(e_));          \
      if (e_ == cudaErrorCooperativeLaunchTooLarge)                                      \
        return jfail(CONCORD_E_OCCUPANCY, "%s: %s", #expr, cudaGetErrorString(e_));      \
      return jfail(CONCORD_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
    }                                                                                    \
  } while (0)

constexpr int kJHistCap = 8192;

}  // namespace

struct concord_joint {
  int device = -1, sms = 0;
  int p = 0, P = 0, ld = 0, precision = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  double *S64[2] = {}, *W64[2] = {}, *Om64[2] = {};
  float *S32[2] = {}, *W32[2] = {}, *Om32[2] = {};  // mixed precision only
  bool have_S[2] = {false, false};
  bool f32_current = false;  // the latest iterate lives in the FP32 arrays
  unsigned* barrier = nullptr;
  unsigned* row_ver = nullptr;  // [p] row versions of the dataflow colour loop
  int variant = CONCORD_JOINT_ROWFLAGS;
  int* abort_info = nullptr;  // [0] abort word, [1] vertex, [2] step
  int* bad = nullptr;
  double* scratch = nullptr;  // p doubles (diagonal checks)
  double* partials = nullptr;
  double* hist = nullptr;
  double* result = nullptr;
  double* h_result = nullptr;  // pinned: kJRes doubles, then 3 ints of abort info, then bad
  double timeout_s = 2.0;
  int fault_row = -1, fault_step = -1;  // one-shot failure-testing switch
  int grid_override = 0;
  int hist_rows = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

bool mixed(const concord_joint* jt) { return jt->precision == CONCORD_MIXED; }

int default_grid(const concord_joint* jt) {
  if (jt->grid_override > 0) return jt->grid_override < jt->sms ? jt->grid_override : jt->sms;
  // every SM: the colour steps are latency-bound chains, and more warps in
  // flight shorten them (measured at p = 1000: 50.2 ms with one CTA per 16
  // pairs of a colour, 43.6 ms with one CTA per SM)
  return jt->sms;
}

void free_all(concord_joint* jt) {
  void* dev[] = {jt->S64[0], jt->S64[1], jt->W64[0], jt->W64[1], jt->Om64[0], jt->Om64[1],
                 jt->S32[0], jt->S32[1], jt->W32[0], jt->W32[1], jt->Om32[0], jt->Om32[1],
                 jt->barrier,  jt->row_ver,    jt->abort_info, jt->bad, jt->scratch, jt->partials,
                 jt->hist,     jt->result};
  for (void* d : dev)
    if (d) cudaFree(d);
  if (jt->h_result) cudaFreeHost(jt->h_result);
  if (jt->ev0) cudaEventDestroy(jt->ev0);
  if (jt->ev1) cudaEventDestroy(jt->ev1);
  if (jt->own_stream) cudaStreamDestroy(jt->own_stream);
}

// Copy the FP32 iterate into the FP64 arrays (mixed: promotion before the
// FP64 phase, or a readout) and rebuild W64 from it.
int promote(concord_joint* jt) {
  if (!jt->f32_current) return CONCORD_OK;
  for (int m = 0; m < 2; ++m) {
    JCK(launch_convert(jt->Om32[m], 1, jt->ld, jt->Om64[m], 0, jt->ld, jt->p, jt->p, jt->stream));
    JCK(launch_joint_refresh(jt->Om64[m], jt->S64[m], jt->W64[m], jt->p, jt->ld, false,
                             jt->stream));
  }
  jt->f32_current = false;
  return CONCORD_OK;
}

// The FP64 iterate into the FP32 arrays (mixed: before an FP32 phase).
int demote(concord_joint* jt) {
  if (jt->f32_current) return CONCORD_OK;
  for (int m = 0; m < 2; ++m) {
    JCK(launch_convert(jt->Om64[m], 0, jt->ld, jt->Om32[m], 1, jt->ld, jt->p, jt->p, jt->stream));
    JCK(launch_joint_refresh(jt->Om32[m], jt->S32[m], jt->W32[m], jt->p, jt->ld, true,
                             jt->stream));
  }
  jt->f32_current = true;
  return CONCORD_OK;
}

struct PhaseOut {
  int sweeps = 0, status = 0, first_delta = 0;
  double kkt = 0, obj = 0, delta = 0, moved = 0;
  int timeout_where = 0, timeout_step = -1;  // on a wait that ran out: row (>= 0) or -1 - CTA
};

// One persistent launch in precision T (f32 selects the FP32 arrays).
int run_phase(concord_joint* jt, bool f32, double l1, double l2, double tol, int n_sweeps,
              bool stall_stop, bool eval_first, PhaseOut* out) {
  const int grid = default_grid(jt);
  int bps = 0;
  JCK(joint_occupancy(f32, &bps));
  if (bps < 1 || grid > bps * jt->sms)
    return jfail(CONCORD_E_OCCUPANCY, "joint sweep: %d CTAs cannot be co-resident", grid);
  if ((long long)n_sweeps * jt->P >= (1ll << 31))
    return jfail(CONCORD_E_ARG, "n_sweeps x colours must stay below 2^31 per launch");
  JCK(cudaMemsetAsync(jt->barrier, 0, sizeof(unsigned), jt->stream));
  unsigned* rv = jt->variant == CONCORD_JOINT_ROWFLAGS ? jt->row_ver : nullptr;
  if (rv) JCK(cudaMemsetAsync(rv, 0, sizeof(unsigned) * jt->p, jt->stream));
  JCK(cudaMemsetAsync(jt->abort_info, 0, 3 * sizeof(int), jt->stream));
  WaitCtl w;
  w.abort = jt->abort_info;
  w.info = jt->abort_info + 1;
  w.timeout_ns = (uint64_t)(jt->timeout_s * 1e9);
  const int hist_left = kJHistCap - jt->hist_rows;
  const int fault_row = rv ? jt->fault_row : -1, fault_step = rv ? jt->fault_step : -1;
  jt->fault_row = -1;  // one-shot
  jt->fault_step = -1;
  if (f32) {
    JointArgs<float> a{};
    a.p = jt->p;
    a.P = jt->P;
    a.ld = jt->ld;
    for (int m = 0; m < 2; ++m) {
      a.S[m] = jt->S32[m];
      a.W[m] = jt->W32[m];
      a.Om[m] = jt->Om32[m];
    }
    a.lambda1 = l1;
    a.lambda2 = l2;
    a.tol = tol;
    a.delta_tol = 1e-5;
    a.n_sweeps = n_sweeps;
    a.stall_stop = stall_stop ? 1 : 0;
    a.eval_first = eval_first ? 1 : 0;
    a.barrier = jt->barrier;
    a.row_ver = rv;
    a.wait = w;
    a.fault_row = fault_row;
    a.fault_step = fault_step;
    a.partials = jt->partials;
    a.hist = jt->hist + (size_t)jt->hist_rows * kJHist;
    a.hist_len = hist_left > 0 ? hist_left : 0;
    a.result = jt->result;
    JCK(launch_joint(a, grid, jt->stream));
  } else {
    JointArgs<double> a{};
    a.p = jt->p;
    a.P = jt->P;
    a.ld = jt->ld;
    for (int m = 0; m < 2; ++m) {
      a.S[m] = jt->S64[m];
      a.W[m] = jt->W64[m];
      a.Om[m] = jt->Om64[m];
    }
    a.lambda1 = l1;
    a.lambda2 = l2;
    a.tol = tol;
    a.delta_tol = 1e-5;
    a.n_sweeps = n_sweeps;
    a.stall_stop = stall_stop ? 1 : 0;
    a.eval_first = eval_first ? 1 : 0;
    a.barrier = jt->barrier;
    a.row_ver = rv;
    a.wait = w;
    a.fault_row = fault_row;
    a.fault_step = fault_step;
    a.partials = jt->partials;
    a.hist = jt->hist + (size_t)jt->hist_rows * kJHist;
    a.hist_len = hist_left > 0 ? hist_left : 0;
    a.result = jt->result;
    JCK(launch_joint(a, grid, jt->stream));
  }
  JCK(cudaMemcpyAsync(jt->h_result, jt->result, kJRes * sizeof(double), cudaMemcpyDeviceToHost,
                      jt->stream));
  int* h_abort = reinterpret_cast<int*>(jt->h_result + kJRes);
  JCK(cudaMemcpyAsync(h_abort, jt->abort_info, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                      jt->stream));
  JCK(cudaStreamSynchronize(jt->stream));
  const double* r = jt->h_result;
  out->sweeps = (int)r[kJResSweeps];
  out->kkt = r[kJResKkt];
  out->obj = r[kJResObj];
  out->delta = r[kJResDelta];
  out->moved = r[kJResMoved];
  out->status = (int)r[kJResStatus];
  out->first_delta = (int)r[kJResFirstDelta];
  jt->hist_rows += out->sweeps < hist_left ? out->sweeps : (hist_left > 0 ? hist_left : 0);
  if (h_abort[0] != 0 || out->status == kJStatusAborted) {
    out->timeout_where = h_abort[1];
    out->timeout_step = h_abort[2];
    if (h_abort[1] >= 0)
      return jfail(CONCORD_E_TIMEOUT,
                   "joint sweep: the wait for row %d ran out (colour step %d)", h_abort[1],
                   h_abort[2]);
    return jfail(CONCORD_E_TIMEOUT, "joint sweep: a grid barrier wait ran out (CTA %d, step %d)",
                 -1 - h_abort[1], h_abort[2]);
  }
  return CONCORD_OK;
}

int check_ready(concord_joint* jt) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (!jt->have_S[0] || !jt->have_S[1])
    return jfail(CONCORD_E_ARG, "both populations' S must be set first");
  return CONCORD_OK;
}

int check_lambdas(double l1, double l2) {
  if (!(l1 >= 0.0) || !(l2 >= 0.0) || !isfinite(l1) || !isfinite(l2))
    return jfail(CONCORD_E_ARG, "lambda1 and lambda2 must be finite and >= 0");
  return CONCORD_OK;
}

void fill_result(concord_result* res, const PhaseOut& o, int sweeps, int sweeps32, double l1,
                 int first_delta, double seconds, int status) {
  if (!res) return;
  memset(res, 0, sizeof *res);
  res->status = status;
  res->sweeps = sweeps;
  res->sweeps_fp32 = sweeps32;
  res->first_delta_sweep = first_delta;
  res->objective = o.obj;
  res->kkt = o.kkt;
  res->delta = o.delta;
  res->lambda = l1;
  res->active_pairs = (long long)o.moved;
  res->seconds = seconds;
  res->timeout_vertex = -1;
  res->timeout_step = -1;
  if (status == CONCORD_E_TIMEOUT) {
    res->timeout_vertex = o.timeout_where;
    res->timeout_step = o.timeout_step;
  }
}

int map_status(const PhaseOut& o) {
  switch (o.status) {
    case kJStatusConverged: return CONCORD_OK;
    case kJStatusNonfinite:
      return jfail(CONCORD_E_NONFINITE, "joint sweep: non-finite KKT residual or objective");
    default: return CONCORD_NOT_CONVERGED;
  }
}

}  // namespace

extern "C" {

int concord_joint_create(concord_joint** out, int p, int precision, int device) {
  if (!out) return jfail(CONCORD_E_ARG, "out is NULL");
  *out = nullptr;
  if (p < 2) return jfail(CONCORD_E_ARG, "p must be >= 2 (got %d)", p);
  if (precision != CONCORD_FP64 && precision != CONCORD_MIXED)
    return jfail(CONCORD_E_ARG, "precision must be CONCORD_FP64 or CONCORD_MIXED");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return jfail(CONCORD_E_CUDA, "no CUDA device");
  if (device < 0) JCK(cudaGetDevice(&device));
  if (device >= ndev) return jfail(CONCORD_E_ARG, "device %d out of range", device);
  JCK(cudaSetDevice(device));
  cudaDeviceProp prop;
  JCK(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return jfail(CONCORD_E_CUDA, "library is built for sm_103a; device is sm_%d%d", prop.major,
                 prop.minor);
  if (!prop.cooperativeLaunch) return jfail(CONCORD_E_CUDA, "device lacks cooperative launch");
  concord_joint* jt = new concord_joint();
  jt->device = device;
  jt->sms = prop.multiProcessorCount;
  jt->p = p;
  jt->P = p + (p & 1) - 1;
  jt->ld = (p + 31) / 32 * 32;
  jt->precision = precision;
  const size_t mat = (size_t)p * jt->ld;
  int rc = CONCORD_OK;
#define JALLOC(ptr, bytes)                                                      \
  do {                                                                          \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                       \
    if (e_ != cudaSuccess) {                                                    \
      rc = jfail(CONCORD_E_NOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes),       \
                 cudaGetErrorString(e_));                                       \
      goto fail_out;                                                            \
    }                                                                           \
  } while (0)
  {
    if (cudaStreamCreateWithFlags(&jt->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = jfail(CONCORD_E_CUDA, "cudaStreamCreate failed");
      goto fail_out;
    }
    jt->stream = jt->own_stream;
    for (int m = 0; m < 2; ++m) {
      JALLOC(jt->S64[m], mat * 8);
      JALLOC(jt->W64[m], mat * 8);
      JALLOC(jt->Om64[m], mat * 8);
      if (precision == CONCORD_MIXED) {
        JALLOC(jt->S32[m], mat * 4);
        JALLOC(jt->W32[m], mat * 4);
        JALLOC(jt->Om32[m], mat * 4);
      }
    }
    JALLOC(jt->barrier, sizeof(unsigned));
    JALLOC(jt->row_ver, sizeof(unsigned) * p);
    JALLOC(jt->abort_info, 3 * sizeof(int));
    JALLOC(jt->bad, sizeof(int));
    JALLOC(jt->scratch, sizeof(double) * p);
    JALLOC(jt->partials, sizeof(double) * 2 * jt->sms * kJParts);
    JALLOC(jt->hist, sizeof(double) * kJHistCap * kJHist);
    JALLOC(jt->result, sizeof(double) * kJRes);
    if (cudaMallocHost((void**)&jt->h_result, sizeof(double) * (kJRes + 4)) != cudaSuccess) {
      rc = jfail(CONCORD_E_NOMEM, "cudaMallocHost failed");
      goto fail_out;
    }
    if (cudaEventCreate(&jt->ev0) != cudaSuccess || cudaEventCreate(&jt->ev1) != cudaSuccess) {
      rc = jfail(CONCORD_E_CUDA, "cudaEventCreate failed");
      goto fail_out;
    }
  }
#undef JALLOC
  *out = jt;
  return CONCORD_OK;
fail_out:
  free_all(jt);
  delete jt;
  return rc;
}

int concord_joint_destroy(concord_joint* jt) {
  if (!jt) return CONCORD_OK;
  cudaSetDevice(jt->device);
  if (jt->stream) cudaStreamSynchronize(jt->stream);
  free_all(jt);
  delete jt;
  return CONCORD_OK;
}

int concord_joint_set_stream(concord_joint* jt, void* stream) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  jt->stream = stream ? (cudaStream_t)stream : jt->own_stream;
  return CONCORD_OK;
}

int concord_joint_set_timeout(concord_joint* jt, double seconds) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (!(seconds > 0.0) || seconds > 3600.0)
    return jfail(CONCORD_E_ARG, "timeout must be in (0, 3600] s");
  jt->timeout_s = seconds;
  return CONCORD_OK;
}

int concord_joint_set_fault(concord_joint* jt, int row, int step) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (row >= jt->p) return jfail(CONCORD_E_ARG, "row must be < p (or < 0 to clear)");
  if (row >= 0 && step < 0) return jfail(CONCORD_E_ARG, "step must be >= 0");
  jt->fault_row = row < 0 ? -1 : row;
  jt->fault_step = row < 0 ? -1 : step;
  return CONCORD_OK;
}

int concord_joint_set_variant(concord_joint* jt, int variant) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (variant != CONCORD_JOINT_ROWFLAGS && variant != CONCORD_JOINT_BARRIER)
    return jfail(CONCORD_E_ARG, "variant must be CONCORD_JOINT_ROWFLAGS or CONCORD_JOINT_BARRIER");
  jt->variant = variant;
  return CONCORD_OK;
}

int concord_joint_set_grid(concord_joint* jt, int ctas) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (ctas < 0) return jfail(CONCORD_E_ARG, "ctas must be >= 0");
  jt->grid_override = ctas;
  return CONCORD_OK;
}

int concord_joint_set_S(concord_joint* jt, int m, const void* S_dev, int s_dtype, int lds) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (m != 0 && m != 1) return jfail(CONCORD_E_ARG, "population must be 0 or 1");
  if (!S_dev) return jfail(CONCORD_E_ARG, "S is NULL");
  if (s_dtype != CONCORD_F64 && s_dtype != CONCORD_F32)
    return jfail(CONCORD_E_ARG, "s_dtype must be CONCORD_F64 or CONCORD_F32");
  if (lds < jt->p) return jfail(CONCORD_E_ARG, "lds < p");
  JCK(cudaSetDevice(jt->device));
  const int f32 = s_dtype == CONCORD_F32;
  JCK(launch_convert(S_dev, f32, lds, jt->S64[m], 0, jt->ld, jt->p, jt->p, jt->stream));
  JCK(cudaMemsetAsync(jt->bad, 0, sizeof(int), jt->stream));
  JCK(launch_extract_diag(jt->S64[m], 0, jt->ld, jt->p, jt->scratch, nullptr, 0, jt->bad,
                          jt->stream));
  JCK(launch_check_symmetric(jt->S64[m], 0, jt->p, jt->ld, jt->bad, jt->stream));
  int* hb = reinterpret_cast<int*>(jt->h_result + kJRes) + 3;
  JCK(cudaMemcpyAsync(hb, jt->bad, sizeof(int), cudaMemcpyDeviceToHost, jt->stream));
  JCK(cudaStreamSynchronize(jt->stream));
  if (*hb != 0) {
    jt->have_S[m] = false;
    return jfail((*hb & 2) ? CONCORD_E_NONFINITE : ((*hb & 1) ? CONCORD_E_NONPOS_DIAG
                                                             : CONCORD_E_ARG),
                 "S of population %d: %s", m,
                 (*hb & 2) ? "non-finite entry" : "non-positive diagonal or not symmetric");
  }
  if (mixed(jt))
    JCK(launch_convert(jt->S64[m], 0, jt->ld, jt->S32[m], 1, jt->ld, jt->p, jt->p, jt->stream));
  // Omega_m = I, W_m = S_m; the other population's iterate moves to FP64
  JCK(launch_set_identity(jt->Om64[m], 0, jt->p, jt->ld, jt->stream));
  JCK(cudaMemcpyAsync(jt->W64[m], jt->S64[m], sizeof(double) * jt->p * jt->ld,
                      cudaMemcpyDeviceToDevice, jt->stream));
  if (mixed(jt)) {
    int o = 1 - m;
    if (jt->f32_current && jt->have_S[o]) {
      JCK(launch_convert(jt->Om32[o], 1, jt->ld, jt->Om64[o], 0, jt->ld, jt->p, jt->p,
                         jt->stream));
      JCK(launch_joint_refresh(jt->Om64[o], jt->S64[o], jt->W64[o], jt->p, jt->ld, false,
                               jt->stream));
    }
    jt->f32_current = false;
  }
  jt->have_S[m] = true;
  JCK(cudaStreamSynchronize(jt->stream));
  return CONCORD_OK;
}

int concord_joint_set_omega(concord_joint* jt, int m, const void* Om_dev, int dtype, int ld) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (m != 0 && m != 1) return jfail(CONCORD_E_ARG, "population must be 0 or 1");
  if (!jt->have_S[m]) return jfail(CONCORD_E_ARG, "S of population %d is not set", m);
  if (!Om_dev) return jfail(CONCORD_E_ARG, "Omega is NULL");
  if (dtype != CONCORD_F64 && dtype != CONCORD_F32)
    return jfail(CONCORD_E_ARG, "dtype must be CONCORD_F64 or CONCORD_F32");
  if (ld < jt->p) return jfail(CONCORD_E_ARG, "ld < p");
  JCK(cudaSetDevice(jt->device));
  int rc = promote(jt);
  if (rc != CONCORD_OK) return rc;
  JCK(launch_convert(Om_dev, dtype == CONCORD_F32, ld, jt->Om64[m], 0, jt->ld, jt->p, jt->p,
                     jt->stream));
  JCK(cudaMemsetAsync(jt->bad, 0, sizeof(int), jt->stream));
  JCK(launch_extract_diag(jt->Om64[m], 0, jt->ld, jt->p, jt->scratch, nullptr, 0, jt->bad,
                          jt->stream));
  JCK(launch_check_symmetric(jt->Om64[m], 0, jt->p, jt->ld, jt->bad, jt->stream));
  int* hb = reinterpret_cast<int*>(jt->h_result + kJRes) + 3;
  JCK(cudaMemcpyAsync(hb, jt->bad, sizeof(int), cudaMemcpyDeviceToHost, jt->stream));
  JCK(cudaStreamSynchronize(jt->stream));
  if (*hb != 0) {
    JCK(launch_set_identity(jt->Om64[m], 0, jt->p, jt->ld, jt->stream));
    JCK(cudaMemcpyAsync(jt->W64[m], jt->S64[m], sizeof(double) * jt->p * jt->ld,
                        cudaMemcpyDeviceToDevice, jt->stream));
    JCK(cudaStreamSynchronize(jt->stream));
    return jfail((*hb & 2) ? CONCORD_E_NONFINITE : CONCORD_E_ARG,
                 "Omega of population %d: %s (reset to I)", m,
                 (*hb & 2) ? "non-finite entry" : "non-positive diagonal or not symmetric");
  }
  JCK(launch_joint_refresh(jt->Om64[m], jt->S64[m], jt->W64[m], jt->p, jt->ld, false,
                           jt->stream));
  JCK(cudaStreamSynchronize(jt->stream));
  return CONCORD_OK;
}

int concord_joint_get_omega(concord_joint* jt, int m, void* Om_dev, int dtype, int ld) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (m != 0 && m != 1) return jfail(CONCORD_E_ARG, "population must be 0 or 1");
  if (!Om_dev) return jfail(CONCORD_E_ARG, "Omega is NULL");
  if (dtype != CONCORD_F64 && dtype != CONCORD_F32)
    return jfail(CONCORD_E_ARG, "dtype must be CONCORD_F64 or CONCORD_F32");
  if (ld < jt->p) return jfail(CONCORD_E_ARG, "ld < p");
  JCK(cudaSetDevice(jt->device));
  if (jt->f32_current)
    JCK(launch_convert(jt->Om32[m], 1, jt->ld, Om_dev, dtype == CONCORD_F32, ld, jt->p, jt->p,
                       jt->stream));
  else
    JCK(launch_convert(jt->Om64[m], 0, jt->ld, Om_dev, dtype == CONCORD_F32, ld, jt->p, jt->p,
                       jt->stream));
  JCK(cudaStreamSynchronize(jt->stream));
  return CONCORD_OK;
}

int concord_joint_sweep(concord_joint* jt, double lambda1, double lambda2, int n_sweeps,
                        concord_result* res) {
  int rc = check_ready(jt);
  if (rc != CONCORD_OK) return rc;
  if ((rc = check_lambdas(lambda1, lambda2)) != CONCORD_OK) return rc;
  if (n_sweeps < 0) return jfail(CONCORD_E_ARG, "n_sweeps must be >= 0");
  JCK(cudaSetDevice(jt->device));
  jt->hist_rows = 0;
  const bool f32 = mixed(jt);
  if (f32 && (rc = demote(jt)) != CONCORD_OK) return rc;
  JCK(cudaEventRecord(jt->ev0, jt->stream));
  PhaseOut o;
  rc = run_phase(jt, f32, lambda1, lambda2, 0.0, n_sweeps, false, false, &o);
  if (rc == CONCORD_E_TIMEOUT) fill_result(res, o, o.sweeps, f32 ? o.sweeps : 0, lambda1, 0, 0.0, rc);
  if (rc != CONCORD_OK) return rc;
  JCK(cudaEventRecord(jt->ev1, jt->stream));
  JCK(cudaEventSynchronize(jt->ev1));
  float ms = 0.f;
  JCK(cudaEventElapsedTime(&ms, jt->ev0, jt->ev1));
  const int st = o.status == kJStatusNonfinite ? map_status(o) : CONCORD_OK;
  fill_result(res, o, o.sweeps, f32 ? o.sweeps : 0, lambda1, o.first_delta, ms * 1e-3, st);
  return st;
}

int concord_joint_run(concord_joint* jt, double lambda1, double lambda2, double tol,
                      int max_sweeps, concord_result* res) {
  int rc = check_ready(jt);
  if (rc != CONCORD_OK) return rc;
  if ((rc = check_lambdas(lambda1, lambda2)) != CONCORD_OK) return rc;
  if (!(tol > 0.0)) return jfail(CONCORD_E_ARG, "tol must be > 0");
  if (max_sweeps < 0) return jfail(CONCORD_E_ARG, "max_sweeps must be >= 0");
  JCK(cudaSetDevice(jt->device));
  jt->hist_rows = 0;
  JCK(cudaEventRecord(jt->ev0, jt->stream));
  PhaseOut o1, o2;
  int sweeps32 = 0, first_delta = 0;
  if (mixed(jt) && max_sweeps > 0) {
    // FP32 phase: sweeps until the tolerance or the FP32 rounding floor
    if ((rc = demote(jt)) != CONCORD_OK) return rc;
    rc = run_phase(jt, true, lambda1, lambda2, tol, max_sweeps, true, true, &o1);
    if (rc == CONCORD_E_TIMEOUT) fill_result(res, o1, o1.sweeps, o1.sweeps, lambda1, 0, 0.0, rc);
    if (rc != CONCORD_OK) return rc;
    if (o1.status == kJStatusNonfinite) return map_status(o1);
    sweeps32 = o1.sweeps;
    first_delta = o1.first_delta;
    if ((rc = promote(jt)) != CONCORD_OK) return rc;
  }
  // FP64 phase (the polish of a mixed solve): the KKT residual is measured in
  // FP64 before any sweep, so an FP32 result that already meets tol is kept
  if ((rc = promote(jt)) != CONCORD_OK) return rc;
  const int left = max_sweeps - sweeps32;
  rc = run_phase(jt, false, lambda1, lambda2, tol, left > 0 ? left : 0, false, true, &o2);
  if (rc == CONCORD_E_TIMEOUT)
    fill_result(res, o2, sweeps32 + o2.sweeps, sweeps32, lambda1, 0, 0.0, rc);
  if (rc != CONCORD_OK) return rc;
  if (!first_delta && o2.first_delta) first_delta = sweeps32 + o2.first_delta;
  JCK(cudaEventRecord(jt->ev1, jt->stream));
  JCK(cudaEventSynchronize(jt->ev1));
  float ms = 0.f;
  JCK(cudaEventElapsedTime(&ms, jt->ev0, jt->ev1));
  const int st = map_status(o2);
  if (o2.sweeps == 0 && sweeps32 > 0) {
    o2.delta = o1.delta;
    o2.moved = o1.moved;
  }
  fill_result(res, o2, sweeps32 + o2.sweeps, sweeps32, lambda1, first_delta, ms * 1e-3, st);
  return st;
}

int concord_joint_get_history(concord_joint* jt, double* hist_host, int max_rows, int* rows) {
  if (!jt) return jfail(CONCORD_E_ARG, "joint state is NULL");
  if (max_rows < 0 || (max_rows > 0 && !hist_host)) return jfail(CONCORD_E_ARG, "bad buffer");
  const int n = jt->hist_rows < max_rows ? jt->hist_rows : max_rows;
  if (n > 0)
    JCK(cudaMemcpy(hist_host, jt->hist, sizeof(double) * n * kJHist, cudaMemcpyDeviceToHost));
  if (rows) *rows = jt->hist_rows;
  return CONCORD_OK;
}

}  // extern "C"
