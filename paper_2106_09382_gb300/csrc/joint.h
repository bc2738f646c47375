// Joint two-population CONCORD (the extension that closes Section 6): kernel
// argument block and launchers.  Internal: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace concord {

constexpr int kJointThreads = 512;               // block size of the joint sweep kernel
constexpr int kJointWarps = kJointThreads / 32;  // pairs a CTA takes per round of a colour

// Per-CTA partials of the fused KKT / objective pass.
constexpr int kJPartKkt = 0, kJPartQuad = 1, kJPartLog = 2, kJPartPen = 3, kJPartFuse = 4,
              kJPartDelta = 5, kJPartMoved = 6;
constexpr int kJParts = 8;

// Result block written by CTA 0.
constexpr int kJResSweeps = 0, kJResKkt = 1, kJResObj = 2, kJResDelta = 3, kJResMoved = 4,
              kJResStatus = 5, kJResFirstDelta = 6;
constexpr int kJRes = 8;
constexpr int kJHist = 4;  // per sweep: delta, kkt, objective, pairs moved

// Status values of kJResStatus.
constexpr int kJStatusConverged = 0, kJStatusMaxSweeps = 1, kJStatusNonfinite = 2,
              kJStatusAborted = 3, kJStatusStalled = 4;
// stall_stop: a sweep that does not bring the KKT residual below 0.9 x the
// best so far counts as stalled; this many in a row end the launch (the FP32
// phase of a mixed solve stops at its rounding floor).
constexpr int kJStallSweeps = 5;

template <typename T>
struct JointArgs {
  int p, P, ld;              // P = colours per sweep (p rounded up to even, minus 1)
  const T* S[2];             // p x ld each, padding columns zero
  T* W[2];                   // W_m = Omega_m S_m (in and out)
  T* Om[2];                  // Omega_m (symmetric; in and out)
  double lambda1, lambda2;   // lasso and fusion weights (S units)
  double tol, delta_tol;     // stop when the joint KKT residual <= tol
  int n_sweeps;              // sweeps this launch may run (0: evaluate only)
  int stall_stop;            // end the launch when the residual stalls (kJStallSweeps)
  int eval_first;            // measure the starting point first (no sweep if it meets tol)
  unsigned* barrier;         // zeroed before the launch
  unsigned* row_ver;         // [p] row versions, zeroed before the launch; nullptr: one grid
                             // barrier per colour step instead
  WaitCtl wait;
  int fault_row = -1, fault_step = -1;  // failure testing (row flags only): row fault_row skips
                              // publishing its version at colour step fault_step of the
                              // launch (counted over all its sweeps); -1: none
  double* partials;          // 2 x gridDim.x x kJParts (double-buffered by sweep parity)
  double* hist;              // hist_len x kJHist
  int hist_len;
  double* result;            // kJRes
};

// One persistent cooperative launch (grid CTAs of kJointThreads threads,
// co-resident): joint sweeps until the stopping rule or n_sweeps.
cudaError_t launch_joint(const JointArgs<double>& a, int grid, cudaStream_t st);
cudaError_t launch_joint(const JointArgs<float>& a, int grid, cudaStream_t st);
cudaError_t joint_occupancy(bool f32, int* blocks_per_sm);

// W (p x ld) = Om S, skipping the zero entries of each row of Om (one warp per
// row, FP64 accumulation); for a warm start.
cudaError_t launch_joint_refresh(const void* Om, const void* S, void* W, int p, int ld, bool f32,
                                 cudaStream_t st);

}  // namespace concord
