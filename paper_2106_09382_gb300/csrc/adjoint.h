// Kernel entry points of the implicit-differentiation pass (adjoint.cu).
// Internal: not part of the C ABI.
#pragma once
#include "kernels.h"

namespace concord {

constexpr int kAdjThreads = 512;
constexpr int kAdjPartPq = 0, kAdjPartRz = 1, kAdjPartRes = 3;  // slots of `partials` (rz, rr / res, dl)
constexpr int kAdjIters = 0, kAdjRel = 1, kAdjTrue = 2, kAdjDlam = 3, kAdjStatus = 4, kAdjBnorm = 5;
constexpr int kAdjRes = 6;
constexpr int kAdjColChunks = 16;  // row chunks of the column sums of dL/dZ

struct AdjArgs {
  int p, ld, nnz;
  const int* rowptr;    // [p + 1] CSR of the active set (diagonal included)
  const int* col;       // [nnz] sorted columns
  const int* erow;      // [nnz] row of each entry
  const int* mirror;    // [nnz] entry (j, i) of entry (i, j)
  const double* om;     // [nnz] Omega on the entries
  const double* S;      // p x ld FP64 S
  const double* minv;   // [nnz] Jacobi preconditioner 1 / H_ee
  const double* b;      // [nnz] right-hand side (both orientations)
  double *x, *r, *z, *pb0, *pb1, *q;  // [nnz] iteration vectors
  double* partials;     // gridDim.x x kParts
  unsigned* barrier;    // zeroed before the launch
  WaitCtl wait;
  double tol;           // stop when ||r|| <= tol ||b||
  int max_iter;
  double* result;       // kAdjRes
};

cudaError_t launch_adj_count(const void* Om, int f32, int p, int ld, int* cnt, int sms,
                             cudaStream_t st);
cudaError_t launch_adj_scan(const int* cnt, int p, int* rowptr, cudaStream_t st);
cudaError_t launch_adj_fill(const void* Om, int f32, int p, int ld, const int* rowptr, int* col,
                            int* erow, double* om, int sms, cudaStream_t st);
cudaError_t launch_adj_prep(int nnz, const int* rowptr, const int* col, const int* erow,
                            const double* om, const double* sdiag, int* mirror, double* minv,
                            int* bad, int sms, cudaStream_t st);
cudaError_t launch_adj_rhs_dense(const void* g, int f32, int ldg, int nnz, const int* col,
                                 const int* erow, double* b, int sms, cudaStream_t st);
// loss (device double) = held-out loss; part: >= part_cap doubles of scratch.
cudaError_t launch_adj_heldout(int nnz, const int* rowptr, const int* col, const int* erow,
                               const int* mirror, const double* om, const void* Sv, int sv_f32,
                               int lds, double* b, double* part, int part_cap, double* loss,
                               int sms, cudaStream_t st);
cudaError_t adj_cg_occupancy(int* blocks_per_sm);
cudaError_t launch_adj_cg(const AdjArgs& a, int grid, cudaStream_t st);
cudaError_t launch_adj_dS(int p, const int* rowptr, const int* col, const double* om,
                          const double* x, double* out, int ldo, int sms, cudaStream_t st);
// dX (n x p, row stride lddx) from the prepared data Z (n x ldz FP64); P, Q,
// dZ: n x ldz scratch; part1/part2: kAdjColChunks x p; m1/m2: p.
cudaError_t launch_adj_data(const double* Z, double* P, double* Q, double* dZ, int ldz, int n, int p,
                            int prep, const int* rowptr, const int* col, const double* om,
                            const double* ah, const double* inv_scale, double* part1, double* part2,
                            double* m1, double* m2, void* dX, int dx_f32, int lddx, int sms,
                            cudaStream_t st);

}  // namespace concord
