/*
 * concord.h -- C ABI of libconcord_gb300.so: CONCORD-PCD (arXiv 2106.09382)
 * on one NVIDIA GB300 (sm_103a).
 *
 * The library estimates a sparse precision matrix Omega by minimising the
 * CONCORD objective (Eq. 1) with the edge-coloured parallel coordinate
 * descent of Algorithm 1:
 *
 *   f(Omega) = - sum_i log w_ii + 1/2 tr(Omega S Omega) + lambda sum_{i<j} |w_ij|
 *
 * written in "S units": S = Z^T Z / n for the n x p data Z after the chosen
 * preparation, so the paper's T = X^T X equals n S and lambda is read on the
 * S scale (the paper's Eq. 1 divided by n, with penalty n * lambda).  The
 * diagonal update (Eq. 2) is the same on either scale.
 *
 * Conventions for every entry point
 *   - Matrices are dense and row-major.  `ld*` arguments are row strides in
 *     elements (>= number of columns).
 *   - `_dev` pointers are device memory on the state's / current device;
 *     `_host` pointers are host memory (pinned or pageable).  The caller owns
 *     every pointer it passes; the library never frees or keeps them after
 *     the call returns (a stream-ordered call has finished reading them once
 *     the stream reaches the call's end).
 *   - Device work is enqueued on the given stream (NULL = the legacy default
 *     stream); calls that return results to host memory synchronise it.
 *   - Every entry point returns a status (CONCORD_OK = 0, > 0 informational,
 *     < 0 error).  On error nothing is written to outputs unless stated, and
 *     concord_last_error() describes the failure (per calling thread).
 *   - Nothing here falls back to a CPU path: without a usable sm_103a device
 *     every call that needs one returns CONCORD_E_CUDA.
 */
#ifndef CONCORD_GB300_H
#define CONCORD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define CONCORD_OK 0
#define CONCORD_NOT_CONVERGED 1     /* max_sweeps reached; outputs are filled */
#define CONCORD_E_ARG (-1)          /* invalid argument (size, pointer, value) */
#define CONCORD_E_NONPOS_DIAG (-2)  /* s_ii <= 0 (constant column) or omega_ii <= 0 */
#define CONCORD_E_NONFINITE (-3)    /* NaN / Inf met in S, Omega or the iteration */
#define CONCORD_E_CUDA (-4)         /* CUDA runtime / launch failure, no device */
#define CONCORD_E_TIMEOUT (-5)      /* a bounded device-side wait ran out */
#define CONCORD_E_NOMEM (-6)        /* device allocation failed */
#define CONCORD_E_OCCUPANCY (-7)    /* persistent grid cannot be co-resident */

/* --------------------------------------------------------------- options */
/* Working precision of a solver state. */
#define CONCORD_FP64 0   /* S, W = Omega S and Omega in FP64 throughout */
#define CONCORD_MIXED 1  /* FP32 S / W / Omega sweeps; FP64 diagonal root,
                            objective and KKT; final FP64 polishing sweeps */

/* Element type of caller buffers. */
#define CONCORD_F64 0
#define CONCORD_F32 1

/* Data preparation applied to X before the Gram (Section 2.1 assumes X
 * centered columnwise; the standardized form also scales every column to
 * unit 1/n variance so that s_ii = 1). */
#define CONCORD_PREP_NONE 0
#define CONCORD_PREP_CENTER 1
#define CONCORD_PREP_STANDARDIZE 2

/* Gram arithmetic. */
#define CONCORD_GRAM_FP64 0    /* FP64 CUDA-core products, FP64 accumulation */
#define CONCORD_GRAM_FP32 1    /* FP32 CUDA-core products, FP32 accumulation */
#define CONCORD_GRAM_TF32X3 2  /* tensor cores (tcgen05, kind::tf32): each FP32
                                  operand split hi + lo, hi*hi + hi*lo + lo*hi,
                                  FP32 accumulation in tensor memory, chunk sums
                                  combined with compensated FP32 (TwoSum);
                                  |dS| <= 128 * 2^-24 + 2^-20 for standardized Z */
#define CONCORD_GRAM_BF16X3 3  /* the same with bf16 hi + lo parts (tcgen05,
                                  kind::f16): half the operand bytes, twice the
                                  MMA rate; |dS| <= 256 * 2^-24 + 2^-14 */

/* Sweep-kernel variant (concord_set_sweep_variant). */
#define CONCORD_SWEEP_AUTO 0     /* screened sweeps; a sweep whose candidate
                                    pairs overflow the screened kernel's lists
                                    runs on the dense kernel (_DENSE layout) */
#define CONCORD_SWEEP_GRID 1     /* dense: every pair of every colour step on a
                                    persistent cooperative grid, one CTA per SM;
                                    partners swap W scalars through an L2 ring */
#define CONCORD_SWEEP_CLUSTER 2  /* dense: one thread-block cluster (up to 16
                                    SMs); partners swap W scalars through
                                    distributed shared memory (lowest latency
                                    per colour) */
#define CONCORD_SWEEP_SCREENED 3 /* screened: only the pairs that can change
                                    (w_ij != 0 or |W_ij + W_ji| > lambda at the
                                    sweep start) are visited, in colour-step
                                    order, by one thread; every other pair is
                                    verified to stay at zero afterwards, and the
                                    sweep is redone with the pairs that fail.
                                    Same iterates as the dense kernels.  Falls
                                    back to the dense kernel like _AUTO. */
#define CONCORD_SWEEP_DENSE 4    /* dense, layout chosen by precision: FP32
                                    cluster when p fits, else grid; FP64 grid */

/* Stopping rule of concord_run / concord_solve*. */
#define CONCORD_STOP_KKT 0    /* KKT residual <= tol (absolute, S units) */
#define CONCORD_STOP_DELTA 1  /* the paper's rule: |Omega^(t)-Omega^(t-1)|_inf < tol
                                 (Algorithm 1, last line) */

/* ------------------------------------------------------------- results */
/* Filled by concord_sweep / concord_run / concord_solve*.  Plain C layout:
 * 4 ints, 4 doubles, 1 int64, 1 double, 9 ints (see concord_result_size). */
typedef struct concord_result {
    int status;            /* CONCORD_OK, CONCORD_NOT_CONVERGED or an error  */
    int sweeps;            /* outer iterations of Algorithm 1 done (all phases) */
    int sweeps_fp32;       /* of which in FP32 (MIXED first phase)            */
    int first_delta_sweep; /* first sweep with delta < delta_tol (0 = never)  */
    double objective;      /* f(Omega) at return, FP64 accumulation           */
    double kkt;            /* KKT residual at return (definition below)       */
    double delta;          /* |Omega^(t) - Omega^(t-1)|_inf of the last sweep */
    double lambda;         /* the lambda used                                  */
    long long active_pairs;/* pairs whose value changed in the last sweep      */
    double seconds;        /* device time of the call (CUDA events)            */
    int timeout_vertex;    /* on CONCORD_E_TIMEOUT: vertex whose wait ran out  */
    int timeout_step;      /*                        and the colour step        */
    int screen_redos;      /* screened sweeps redone after a pair outside the
                              candidates failed the verification */
    int dense_sweeps;      /* sweeps handed from the screened to the dense kernel */
    int s_refined;         /* MIXED: entries of S recomputed in FP64 accuracy
                              before the polish (concord_set_refine); 0 if none */
    int lazy_sweeps;       /* screened sweeps that skipped the verification
                              pass (concord_set_lazy_verify); sparse polish
                              sweeps count as well */
    int sparse_sweeps;     /* MIXED: polish sweeps run by the sparse polish
                              (concord_set_sparse_polish) */
    int partial_sweeps;    /* lazy sweeps (FP32 screened or sparse polish) that
                              verified only the pairs of the rows whose bound
                              left half the margin */
} concord_result;

/* KKT residual (absolute, S units), with W = Omega S and G = W + W^T:
 *   max over i of |W_ii - 1/w_ii|, over i<j with w_ij != 0 of
 *   |G_ij + lambda sign(w_ij)|, and over i<j with w_ij == 0 of
 *   max(|G_ij| - lambda, 0):  the subgradient conditions of Eq. 1. */

/* Size of concord_result in bytes (lets bindings check their layout). */
size_t concord_result_size(void);

/* Text of the last error on the calling thread ("" if none).  The pointer
 * stays valid until the next library call on the same thread. */
const char *concord_last_error(void);

/* Library version string. */
const char *concord_version(void);

/* --------------------------------------------------------------- schedule */
/*
 * concord_schedule -- the circle-method edge colouring of K_p (Section 3.2;
 * Algorithm 1's index rotation; Table 1 shows p = 6).
 *
 * pairs_host: host int32 array of (pe-1) * (pe/2) * 2 elements, pe = p + (p
 *   mod 2).  Entry [(k*(pe/2) + q)*2 + {0,1}] is the 0-based vertex pair of
 *   slot q of colour k, in Algorithm 1's order; the pair that holds the extra
 *   vertex of odd p is written as (-1, -1) (step (iii): it is discarded).
 * n_colours: receives pe - 1 (the minimum by Theorem 1).
 * Host only; needs no device.  Errors: CONCORD_E_ARG if p < 2 or a pointer
 * is NULL.
 */
int concord_schedule(int p, int32_t *pairs_host, int *n_colours);

/* ------------------------------------------------------------------ gram */
/*
 * concord_gram -- S = Z^T Z / n (Algorithm 1, T <- X^T X, divided by n),
 * Z = X after `prep` (Section 2.1: columns centered; STANDARDIZE also scales
 * them to unit 1/n variance).
 *
 * X_dev: n x p, row stride ldx, element type x_dtype (F64 or F32); not
 *   modified.
 * S_dev: p x p output, row stride lds, element type s_dtype; both triangles
 *   are written, exactly symmetric.  Must not overlap X_dev.
 * mode: CONCORD_GRAM_FP64 / _FP32 / _TF32X3.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Scratch memory is allocated and freed inside the call (stream-ordered).
 * Errors: CONCORD_E_ARG (n < 1, p < 2, ld too small, NULL),
 *   CONCORD_E_NONPOS_DIAG (a constant column under STANDARDIZE, detected on
 *   the device and reported after a stream synchronisation),
 *   CONCORD_E_NOMEM, CONCORD_E_CUDA.
 */
int concord_gram(const void *X_dev, int x_dtype, int n, int p, int ldx, int prep,
                 int mode, void *S_dev, int s_dtype, int lds, void *stream);

/*
 * concord_gram_static -- the same S = Z^T Z / n as concord_gram in
 * CONCORD_GRAM_FP64 mode (Z = X after `prep`; FP64 products and sums; S is
 * FP64, p x p, row stride lds, both triangles written), but without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory while they
 * run -- a framework that owns all device memory through its own pool, a
 * latency-critical loop in which cudaMalloc / cudaFree would synchronise the
 * device, or a deployment that forbids dynamic allocation after start-up.
 *
 * X is standardized while the tiles are staged, and the per-column
 * statistics live in a fixed device array of the library (2 x 16384 doubles
 * plus a status word, held on every device that loads the library until the
 * process exits).  Hence:
 *   - p must be <= 16384; larger p returns CONCORD_E_ARG (use concord_gram);
 *   - the first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and caches it; make that
 *     first call on each device before any stream capture begins;
 *   - every call shares the array and it keeps the last call's contents;
 *     the status word is cleared by each call; calls that overlap on the GPU
 *     (different streams or host threads at the same time) race on it and
 *     must be serialised by the caller.
 * Every call waits for `stream` to finish its work, then reads the status
 * word back to report a constant or non-finite column.
 * Errors: CONCORD_E_ARG, CONCORD_E_NONPOS_DIAG, CONCORD_E_NONFINITE,
 * CONCORD_E_CUDA.
 */
int concord_gram_static(const void *X_dev, int x_dtype, int n, int p, int ldx, int prep,
                        double *S_dev, int lds, void *stream);

/* ----------------------------------------------------------- solver state */
typedef struct concord_state concord_state;

/*
 * concord_create -- allocate a solver for dimension p (>= 2) on `device`
 * (-1 = current device) in `precision` (CONCORD_FP64 or CONCORD_MIXED).
 * n_cap (>= 0) reserves room for data with up to n_cap rows, used by
 * concord_solve_device / concord_solve_host (0 = none; the data path then
 * returns CONCORD_E_ARG).
 *
 * Device memory held (ld = p rounded up to a multiple of 32 elements,
 * e = 4 for MIXED, 8 for FP64):  S, W = Omega S, Omega: 3 p ld e bytes, plus
 * for MIXED the FP64 polishing copies 3 p ld 8 bytes, plus small per-vertex
 * and per-block arrays and the data workspace.  Omega starts at I.
 * The state owns one CUDA stream unless concord_set_stream gives another.
 * Errors: CONCORD_E_ARG, CONCORD_E_NOMEM, CONCORD_E_CUDA.
 */
int concord_create(concord_state **out, int p, int precision, int n_cap, int device);

/* Free every device and host resource of the state (NULL is accepted). */
int concord_destroy(concord_state *st);

/* Use `stream` (a cudaStream_t, NULL = the state's own stream) for all
 * later work on the state. */
int concord_set_stream(concord_state *st, void *stream);

/* Upper bound, in seconds (> 0), on every device-side wait (per-vertex
 * mailboxes, grid barriers).  A wait that runs out sets CONCORD_E_TIMEOUT,
 * the kernel returns and the context stays usable.  Default 2 s. */
int concord_set_timeout(concord_state *st, double seconds);

/*
 * concord_set_S -- load S (p x p, row stride lds, element type s_dtype,
 * device memory) into the state, converting to the working precision, and
 * reset Omega to I and W to S.  S must be symmetric with s_ii > 0 (checked
 * on the diagonal: CONCORD_E_NONPOS_DIAG / CONCORD_E_NONFINITE).
 */
int concord_set_S(concord_state *st, const void *S_dev, int s_dtype, int lds);

/*
 * concord_set_omega -- warm start (Algorithm 1 takes Omega^(0) as input):
 * copy Omega0 (p x p, device, row stride ld, element type dtype; symmetric,
 * positive diagonal) into the state and recompute W = Omega S.
 * Errors: CONCORD_E_ARG (not symmetric), CONCORD_E_NONPOS_DIAG.
 */
int concord_set_omega(concord_state *st, const void *Omega0_dev, int dtype, int ld);

/* Copy the current Omega (or W = Omega S, or S) of the state out, converted
 * to `dtype`, into device memory with row stride ld. */
int concord_get_omega(concord_state *st, void *Omega_dev, int dtype, int ld);

/*
 * concord_get_omega_csr -- the current Omega (FP64 iterate) in compressed
 * sparse rows, into host (or device) buffers: rowptr[p + 1], col[nnz] (sorted
 * within each row, diagonal included) and val[nnz] (FP64).  The estimate is
 * sparse, so this moves (p + 1) * 4 + nnz * 12 bytes instead of p * p * 8.
 * cap: capacity of col / val in entries; *nnz receives the entry count even
 * when it exceeds cap (then only rowptr is written and CONCORD_E_ARG is
 * returned, so a caller can size its buffers and call again).  The copies
 * are made with cudaMemcpyAsync on the state's stream, which is
 * synchronised before returning.
 */
int concord_get_omega_csr(concord_state *st, int32_t *rowptr, int32_t *col, double *val,
                          int64_t cap, int64_t *nnz);
int concord_get_W(concord_state *st, void *W_dev, int dtype, int ld);

/*
 * concord_get_history -- per-sweep record of the last concord_sweep /
 * concord_run / concord_solve_* on the state: hist_host receives up to
 * max_rows rows of 4 doubles (delta, KKT residual, objective, pairs whose
 * value changed), one per sweep in order (FP32 sweeps first for MIXED);
 * *rows receives the number of sweeps recorded.  hist_host may be NULL to
 * query *rows only.
 */
int concord_get_history(concord_state *st, double *hist_host, int max_rows, int *rows);

/*
 * concord_get_timing -- device time of each persistent sweep-kernel launch
 * of the last concord_sweep / concord_run / concord_solve_* (CUDA events
 * recorded on the state's stream around the launch): launch_ms[q] in
 * milliseconds and launch_sweeps[q] the sweeps it ran, for q < max_launches
 * (MIXED runs launch at least twice: FP32 sweeps, then FP64 polishing; a
 * screened run adds one dense launch per sweep handed to the dense kernel,
 * and the screened launch after it).  Either array
 * may be NULL; *n_launches receives the number of launches (<= 16 recorded).
 */
int concord_get_timing(concord_state *st, double *launch_ms, int *launch_sweeps,
                       int max_launches, int *n_launches);

/* Number of CUDA kernels this library has launched in this process (all
 * states, all entry points): the basis of launch accounting in benchmarks. */
unsigned long long concord_kernel_launches(void);

/*
 * concord_set_sweep_variant -- CONCORD_SWEEP_AUTO (default), _GRID,
 * _CLUSTER, _SCREENED or _DENSE.  The variants compute the same iterates
 * (bit for bit); the dense ones trade latency per colour step (cluster)
 * against memory bandwidth (grid, all SMs); the screened one skips the pairs
 * that stay at zero, which wins whenever few pairs change per sweep.
 * _CLUSTER fails with CONCORD_E_ARG if p exceeds what one cluster holds
 * (cluster size x 512 rows).  Explicit settings (this one and
 * concord_set_rows_per_warp) apply to sweeps in the state's working
 * precision; the FP64 polishing sweeps of a MIXED state use the defaults.
 * concord_get_sweep_variant reports the variant of the last launch and the
 * largest cluster size found (0 = none).  The screened kernel allocates its
 * scratch (two p x p matrices of the FP64 width, candidate lists of
 * max(16 p, 65536) pairs, at most all pairs, with up to max(8 x that, 4M)
 * correction terms) on first use.
 */
int concord_set_sweep_variant(concord_state *st, int variant);
int concord_get_sweep_variant(concord_state *st, int *variant, int *cluster_size);

/*
 * concord_autotune -- picks the sweep kernel and layout for the state's S
 * and a representative lambda by measurement: from Omega = I it runs the
 * solve (concord_run with tol, max_sweeps) once with each of the
 * CONCORD_AUTOTUNE_CHOICES layouts -- the screened kernel; the dense kernel
 * as one cluster at 32, 16, 8, 4 rows per warp; the dense kernel on the grid
 * at 32, 16, 8, 4 rows per warp -- and keeps the one with the least device
 * time per sweep (all launches of the solve).  ms_per_sweep (host,
 * nullable, CONCORD_AUTOTUNE_CHOICES doubles) receives each time, -1 where
 * a layout cannot run at this p; variant / rows_per_warp (nullable) the
 * choice.  Results do not depend on the choice (every layout gives the same
 * iterates).  The state ends at Omega = I.  Synchronises the stream.
 * Errors: CONCORD_E_ARG, CONCORD_E_OCCUPANCY, CONCORD_E_TIMEOUT, CONCORD_E_CUDA.
 */
#define CONCORD_AUTOTUNE_CHOICES 9
int concord_autotune(concord_state *st, double lambda, double tol, int max_sweeps,
                     double *ms_per_sweep, int *variant, int *rows_per_warp);

/*
 * concord_set_poll_sleep -- back-off, in nanoseconds (0..100000), between
 * two polls of a mailbox word in the sweep kernel (__nanosleep); a negative
 * value restores the default (0).  Trades wake-up latency against the load/store
 * bandwidth the polling warps take from the working ones.  Results do not
 * depend on it.
 */
int concord_set_poll_sleep(concord_state *st, int ns);

/*
 * concord_set_rows_per_warp -- work layout of the sweep kernel: each warp
 * owns up to `rows` rows of Omega and W (one row per lane), so `rows` trades
 * scalar efficiency (many rows per warp) against row-update bandwidth (many
 * warps).  0 (default) picks 32 for the cluster variant, 8 for the grid.
 * Results do not depend on it.
 */
int concord_set_rows_per_warp(concord_state *st, int rows);

/*
 * concord_set_gram_mode -- Gram arithmetic used by concord_solve_device /
 * concord_solve_host: CONCORD_GRAM_FP64 (default for FP64 states),
 * CONCORD_GRAM_FP32 or CONCORD_GRAM_TF32X3 (mixed states only; their
 * default).
 */
int concord_set_gram_mode(concord_state *st, int mode);

/*
 * concord_set_refine -- on (1, the default) or off (0): before the FP64
 * polish of a MIXED solve whose S came from data through a reduced-precision
 * Gram (CONCORD_GRAM_TF32X3, _BF16X3, _FP32), recompute in FP64 accuracy the
 * entries of S that the optimality conditions of Eq. 1 read for the pairs
 * that can be active: for every candidate pair (i, j) of the next sweep
 * (w_ij != 0 or |G_ij| > 0.9 lambda) the entries s_kj, k in {i} u N(i), and
 * s_ki, k in {j} u N(j), and for every vertex i the entries s_ki,
 * k in {i} u N(i), where N(i) are the vertices paired with i among the
 * candidates.  They are recomputed from the standardized data rounded to
 * FP32 with compensated (double-float) sums and written into both copies of
 * S kept by the state.  The tensor cores' FP32 accumulation rounds its sums
 * with a bias (on the p = 5000 benchmark workload the 3xTF32 diagonal of S is
 * 1.1e-6 low); with the refinement the polish solves the problem of the exact
 * S instead of the perturbed one.  The count of recomputed entries is
 * reported in concord_result.s_refined.  Results of FP64 states, of states
 * whose S came from concord_set_S and of CONCORD_GRAM_FP64 are unaffected.
 * Errors: CONCORD_E_ARG.
 */
int concord_set_refine(concord_state *st, int on);

/*
 * concord_set_lazy_verify -- on (1, the default) or off (0).  The screened
 * kernel visits only candidate pairs (w_ij != 0 or |G_ij| > 0.9 lambda when
 * the list was screened) and then verifies that no other pair would have
 * left zero, re-screening for the next sweep.  A change d of a candidate
 * (i, u) moves G_ij of a pair outside the list by at most |d| m_u, and a
 * diagonal change by at most |dw| m_i (m_u = max_{x != u} |s_ux|).  While
 * the sum of these bounds since the list was screened stays within 0.09
 * lambda, no pair outside it can reach the threshold, so the sweep skips the
 * verification pass and keeps the list (and its build) for the next sweep.
 * The bound is kept per row (the sum of its changes' bounds since the row's
 * pairs were screened): when only a few rows exceed half the margin,
 * only their pairs are verified and screened (a partial sweep), from the
 * stored rows and their deferred updates.  The iterates are the same either
 * way; concord_result.lazy_sweeps counts the skipped full verifications,
 * partial_sweeps the partial ones among them.  Errors: CONCORD_E_ARG.
 */
int concord_set_lazy_verify(concord_state *st, int on);

/*
 * concord_set_sparse_polish -- on (1, the default) or off (0); CONCORD_MIXED
 * states only (others ignore it).  The FP64 polish of a mixed solve extends
 * the bound of concord_set_lazy_verify across the change from the FP32 to
 * the FP64 S (2 max_i ||Omega_i||_1 max|dS|, dS the refined entries' change
 * or FP32 rounding).  While it holds, the polish sweeps (Eq. 3 and Eq. 2 as
 * their direct sums over the nonzeros of Omega) change only the FP32 phase's
 * last candidates and W = Omega S is never rebuilt in FP64.  A sweep that
 * would break the bound is not committed; W is then rebuilt and the screened
 * polish (which verifies every pair) takes the remaining sweeps.  Compared
 * with the screened polish the iterates agree to FP64 rounding (the sums run
 * in another order).  After a sparse polish the state's FP64 W is rebuilt
 * when it is next needed (concord_get_W, warm starts).
 * Errors: CONCORD_E_ARG.
 */
int concord_set_sparse_polish(concord_state *st, int on);

/*
 * concord_sweep -- run exactly n_sweeps outer iterations of Algorithm 1 at
 * penalty lambda (>= 0) on the state, in its working precision (MIXED: FP32
 * sweeps, no polish):  for colour k = 1..pe-1 all pairs of colour k get the
 * closed-form update of Eq. 3 at once, then every diagonal entry gets Eq. 2;
 * W = Omega S is kept current row by row.  One persistent kernel launch.
 * res (may be NULL) receives the objective, KKT residual and delta after the
 * last sweep.  Synchronises the state's stream.
 */
int concord_sweep(concord_state *st, double lambda, int n_sweeps, concord_result *res);

/*
 * concord_run -- sweeps at lambda until the stopping rule holds (stop_rule
 * CONCORD_STOP_KKT: KKT <= tol; CONCORD_STOP_DELTA: delta < tol) or
 * max_sweeps.  FP64 state: all sweeps in FP64.  MIXED state: FP32 sweeps
 * until the rule holds at max(tol, switch_tol) (switch_tol <= 0 picks
 * max(3 tol, 1e-5)) or until the KKT residual stops falling by 10% for 4
 * sweeps (FP32 rounding floor); then W is rebuilt in FP64 from the FP64
 * copies of S and Omega and FP64 sweeps polish to tol.  Returns CONCORD_OK
 * or CONCORD_NOT_CONVERGED (outputs filled either way) or an error.
 * Synchronises the stream.
 */
int concord_run(concord_state *st, double lambda, double tol, int max_sweeps,
                int stop_rule, double switch_tol, concord_result *res);

/*
 * concord_path -- a warm-started regularisation path (the batched use of
 * Algorithm 1: each lambda is swept from the previous lambda's Omega and W,
 * the first from the state's current iterate).  lambdas (host, n_lambda > 0,
 * each >= 0; usually decreasing from concord_lambda_max) are swept in order
 * until KKT <= tol or max_sweeps per lambda, in the state's working
 * precision (MIXED: FP32 sweeps with the FP64 diagonal, KKT and objective,
 * no FP64 polish; FP64: FP64).  One persistent screened launch walks the
 * whole path; a lambda whose sweeps overflow the candidate lists runs on the
 * dense kernel and the path resumes after it.  results (host, nullable)
 * receives one concord_result per lambda.  omega_out_dev (device, nullable)
 * receives Omega after each lambda: slice k at offset k * p * ld_out, row
 * stride ld_out >= p, element type of the working precision (float for
 * MIXED, double for FP64).  The state ends on the last lambda's iterate.
 */
int concord_path(concord_state *st, const double *lambdas, int n_lambda, double tol,
                 int max_sweeps, concord_result *results, void *omega_out_dev, int ld_out);

/*
 * concord_stability -- stability selection over subsamples: for each of
 * n_sets subsamples of the rows of X (device, n x p, row stride ldx, dtype
 * F64 / F32; subsample b is the set_sizes[b] row indices starting at
 * rows[sum of earlier sizes], host arrays, each size in 2..n_cap), the
 * Gram of its rows (prep as concord_solve_device) and the lambda path over
 * lambdas from Omega = I; freq_dev (device, float, n_lambda x p x p, written
 * completely) receives for each lambda the fraction of subsamples whose
 * Omega has w_ij != 0.  n_workers = 0 (the default) solves every
 * subsample as one problem of a batch (concord_batch_*: one persistent
 * launch per wave of co-resident subsamples, each walking the path, the
 * Gram 3xTF32 for MIXED and FP64 for FP64).  n_workers >= 1 runs that many
 * subsamples concurrently, each on a state of its own (own stream,
 * 1 / n_workers of the SMs, created and destroyed by the call, same
 * precision, n_cap and Gram mode as st) with one host thread; n_workers = 1
 * uses st itself, which then ends on the last subsample's last lambda.
 * Every kernel gives the same iterates and support counts are whole numbers
 * added atomically, so the frequencies agree between the forms whenever no
 * lambda ends on the FP32 stall rule (whose count restarts when the
 * single-state path hands a lambda to the dense kernel).
 */
int concord_stability(concord_state *st, const void *X_dev, int x_dtype, int n, int ldx, int prep,
                      const int *rows, const int *set_sizes, int n_sets, const double *lambdas,
                      int n_lambda, double tol, int max_sweeps, int n_workers, float *freq_dev);


/*
 * concord_solve_device -- the whole path on resident data: prepare X
 * (n <= n_cap rows, device, row stride ldx, x_dtype), S = Z^T Z / n in the
 * state's Gram mode (FP64 state: CONCORD_GRAM_FP64; MIXED:
 * CONCORD_GRAM_TF32X3 then an FP64 copy of the FP32 S for polishing),
 * Omega = I, then concord_run.  Omega_dev (may be NULL) receives
 * Omega in `omega_dtype` with row stride ldo.
 */
int concord_solve_device(concord_state *st, const void *X_dev, int x_dtype, int n,
                         int ldx, int prep, double lambda, double tol, int max_sweeps,
                         int stop_rule, void *Omega_dev, int omega_dtype, int ldo,
                         concord_result *res);

/*
 * concord_solve_host -- as concord_solve_device, with X (n x p, FP64, dense,
 * host) copied in and Omega (p x p, FP64, dense, host) copied out inside the
 * call.  Omega_host may be NULL.
 */
int concord_solve_host(concord_state *st, const double *X_host, int n, int prep,
                       double lambda, double tol, int max_sweeps, int stop_rule,
                       double *Omega_host, concord_result *res);

/*
 * concord_solve -- one-shot convenience: creates a state, solves from host
 * data (is_X != 0: X is n x p; is_X == 0: S is p x p and n is ignored), and
 * destroys the state.  Omega0_host (NULL = I) is an optional warm start.
 */
int concord_solve(const double *data_host, int is_X, int n, int p, int prep,
                  double lambda, double tol, int max_sweeps, int precision,
                  const double *Omega0_host, double *Omega_host, concord_result *res);

/*
 * concord_lambda_max -- max_{i<j} |s_ij| (s_ii^{-1/2} + s_jj^{-1/2}) of the
 * state's S: the smallest lambda at which the diagonal point
 * diag(s_ii^{-1/2}) satisfies the KKT conditions of Eq. 1 (G_ij = s_ij
 * (w_ii + w_jj) there).  Synchronises the stream.
 */
int concord_lambda_max(concord_state *st, double *lambda_max);

/*
 * concord_set_fault -- failure-detection testing.  vertex >= 0 makes that
 * vertex skip publishing its mailbox value at colour step `step` of the next
 * launch, so its partner's bounded wait runs out (CONCORD_E_TIMEOUT with
 * the partner and step in the result).  vertex < 0 clears it.  No kernel
 * faults, traps or hangs: every wait ends at the state's timeout.
 */
int concord_set_fault(concord_state *st, int vertex, int step);

/* ------------------------------------------------ implicit differentiation */
/*
 * Gradients of a loss L(Omega) of the estimate with respect to lambda, S and
 * the data X, by implicit differentiation of the minimiser of Eq. 1.  On the
 * active set A of the state's current Omega (the diagonal and the pairs with
 * w_ij != 0) the subgradient conditions hold with equality,
 *   W_ii - 1/w_ii = 0,   W_ij + W_ji + lambda sign(w_ij) = 0   (W = Omega S),
 * and with A and the signs held fixed (valid when no inactive pair sits on
 * the threshold |W_ij + W_ji| = lambda) they define Omega_A(S, lambda)
 * smoothly.  With b the loss gradient on A (b_ii = dL/dw_ii, b_ij = dL/dw_ij
 * + dL/dw_ji) and H the Hessian of the smooth part of Eq. 1 on A,
 *   (H V)_ij = (V S + S V)_ij,   (H V)_ii = (V S)_ii + v_ii / w_ii^2,
 * the adjoint a = H^{-1} b gives
 *   dL/dlambda = - sum_{i<j in A} a_ij sign(w_ij),
 *   dL/dS      = - Omega Ahat   (Ahat: a as a symmetric matrix on A),
 *   dL/dZ      = Z (dL/dS + dL/dS^T) / n   for S = Z^T Z / n,
 * and dL/dX through the data preparation (Section 2.1).  Gradients with
 * respect to matrices use the full-matrix convention: every entry is an
 * independent variable (a symmetric perturbation of s_ij and s_ji changes L
 * by G_ij + G_ji).  H is applied matrix-free on A (sparse gathers of S, FP64)
 * and the system is solved by Jacobi-preconditioned conjugate gradients in
 * one persistent cooperative launch; no sweep of the solver is stored or
 * replayed.  Everything here is FP64 on the FP64 copy of S; in MIXED
 * precision the FP64 iterate of the last polishing phase is used (after a
 * concord_run / concord_solve_*), else the FP32 iterate widened to FP64.
 *
 * Scratch (allocated on first use, kept by the state): about 84 bytes per
 * entry of A (both orientations of each pair, plus the diagonal) and, for
 * concord_adjoint_data, four n x ld FP64 matrices.
 */

typedef struct concord_adjoint_info {
    int status;            /* CONCORD_OK, or CONCORD_NOT_CONVERGED (max_iter reached) */
    int iterations;        /* conjugate-gradient iterations                        */
    long long active_pairs;/* off-diagonal pairs in A                              */
    double residual;       /* ||b - H a|| / ||b||, recomputed after the last step  */
    double dlambda;        /* dL/dlambda                                           */
    double seconds;        /* device time of the conjugate-gradient launch         */
} concord_adjoint_info;

/*
 * concord_heldout -- the held-out loss of the current Omega,
 *   L = - sum_i log w_ii + 1/2 tr(Omega S_val Omega)
 * (the smooth part of Eq. 1 with a validation Gram S_val = Z_val^T Z_val /
 * n_val), into *loss_host, and its gradient on A as the right-hand side of
 * the next concord_adjoint(st, NULL, ...).  The active set is taken from the
 * current Omega here.  S_val: p x p device, row stride lds (>= p), element
 * type s_dtype; symmetric.  Synchronises the stream.
 * Errors: CONCORD_E_ARG (NULL, lds < p, bad dtype; Omega not symmetric),
 *   CONCORD_E_NONPOS_DIAG (w_ii <= 0), CONCORD_E_NOMEM, CONCORD_E_CUDA.
 */
int concord_heldout(concord_state *st, const void *Sval_dev, int s_dtype, int lds, double *loss_host);

/*
 * concord_adjoint -- solve H a = b on the active set and return dL/dlambda
 * (info->dlambda) and optionally dL/dS.
 * gOmega_dev: dL/dOmega (p x p device, row stride ldg, element type g_dtype,
 *   full-matrix convention); the active set is taken from the current Omega.
 *   NULL: use the gradient left by the last concord_heldout (and its active
 *   set and Omega).
 * tol (> 0): stop when ||b - H a|| <= tol ||b|| (recursive residual);
 *   max_iter >= 1 conjugate-gradient iterations at most.
 * dS_dev: NULL, or p x p FP64 device output (row stride ldds >= p) receiving
 *   dL/dS = -Omega Ahat (every entry written).
 * The adjoint a stays in the state for concord_adjoint_data.  A device wait
 * that runs out returns CONCORD_E_TIMEOUT.  Synchronises the stream.
 * Errors: CONCORD_E_ARG (NULL info, bad sizes, NULL gOmega without a
 *   preceding concord_heldout, Omega not symmetric), CONCORD_E_NONFINITE (H
 *   not positive definite along a search direction, or non-finite values),
 *   CONCORD_E_TIMEOUT, CONCORD_E_NOMEM, CONCORD_E_CUDA.
 */
int concord_adjoint(concord_state *st, const void *gOmega_dev, int g_dtype, int ldg, double tol,
                    int max_iter, double *dS_dev, int ldds, concord_adjoint_info *info);

/*
 * concord_adjoint_data -- dL/dX (n x p device output, row stride lddx,
 * element type dx_dtype) for S = Z^T Z / n, Z = X after `prep`, from the
 * adjoint of the last concord_adjoint.  X_dev: n x p device data (row
 * stride ldx, element type x_dtype), the data S was computed from.  The
 * preparation's statistics are recomputed from X (mean and, for
 * STANDARDIZE, the population standard deviation) and differentiated too.
 * Stream-ordered; synchronises only to report a constant column.
 * Errors: CONCORD_E_ARG (no preceding concord_adjoint, bad sizes),
 *   CONCORD_E_NONPOS_DIAG (constant column under STANDARDIZE),
 *   CONCORD_E_NOMEM, CONCORD_E_CUDA.
 */
int concord_adjoint_data(concord_state *st, const void *X_dev, int x_dtype, int n, int ldx, int prep,
                         void *dX_dev, int dx_dtype, int lddx);

/*
 * concord_tune_lambda -- hypergradient descent on log lambda for the
 * held-out loss of concord_heldout: `steps` times, solve at lambda
 * (concord_run warm-started from the current Omega, KKT <= tol, at most
 * max_sweeps sweeps), take L and dL/dlambda (concord_heldout, then
 * concord_adjoint with cg_tol and at most 10000 iterations), record the row
 *   (lambda, L, dL/dlambda, sweeps, CG iterations, KKT residual)
 * into rows_host[6 k .. 6 k + 5], and move log lambda by
 * -lr * lambda * dL/dlambda.  The state's S is the training Gram.
 * Errors: as concord_run, concord_heldout and concord_adjoint; lambda0 > 0,
 *   steps >= 1, lr >= 0 (CONCORD_E_ARG).
 */
int concord_tune_lambda(concord_state *st, const void *Sval_dev, int s_dtype, int lds, double lambda0,
                        int steps, double lr, double tol, int max_sweeps, double cg_tol,
                        double *rows_host);

/* ------------------------------------ joint two-population CONCORD */
/*
 * The extension that closes Section 6: two precision matrices Omega1, Omega2
 * (one per population, Grams S1, S2 in S units) minimise
 *
 *   sum_m [ - sum_i log w^m_ii + 1/2 tr(Omega_m S_m Omega_m)
 *           + lambda1 sum_{i<j} |w^m_ij| ]
 *   + lambda2 sum_{i<=j} |w^1_ij - w^2_ij|
 *
 * (the joint objective divided by the common n; the fusion penalty covers
 * the diagonal, as the joint objective writes it).  Block coordinate descent
 * moves the pair (w^1_ij, w^2_ij) jointly in Algorithm 1's colour order --
 * blocks of one colour touch disjoint rows, so they are independent as in
 * Lemma 1 -- then the diagonal blocks (w^1_ii, w^2_ii).  Every block update
 * has a closed form: with the sign of the difference fixed the block problem
 * separates into two lasso problems (pairs) or two Eq. 2 roots (diagonal);
 * when neither sign is consistent, the minimiser lies on w^1 = w^2.
 *
 * Joint KKT residual (absolute, S units; the stopping rule): with
 * W_m = Omega_m S_m and, per pair, the smooth gradients G_m = W^m_ij + W^m_ji
 * (diagonal: W^m_ii - 1/w^m_ii), the largest over blocks of
 *   min over admissible u of max(dist(-(G_1 + u), lambda1 d|w^1|),
 *                                dist(-(G_2 - u), lambda1 d|w^2|)),
 * u = lambda2 sign(w^1 - w^2) where the two differ, u in [-lambda2, lambda2]
 * where they are equal (no lasso term on the diagonal).  lambda2 = 0 gives
 * the larger of the two populations' Eq. 1 residuals.
 *
 * Precision: CONCORD_FP64 runs FP64 sweeps; CONCORD_MIXED runs FP32 sweeps
 * (FP64 block arithmetic) until the residual meets tol or stops falling,
 * then FP64 sweeps from the promoted iterate (W rebuilt in FP64).
 *
 * One persistent cooperative launch per phase: colour steps synchronised by
 * per-row version flags (or one grid barrier per colour step), a fused
 * KKT / objective pass after every sweep.
 */
typedef struct concord_joint concord_joint;

/* Allocates the working set for dimension p on `device` (-1 = current): for
 * each population S, W and Omega (p x round_up(p, 32)) in FP64, plus FP32
 * copies under CONCORD_MIXED.  Errors: CONCORD_E_ARG (p < 2, precision),
 * CONCORD_E_CUDA (no sm_103 device), CONCORD_E_NOMEM. */
int concord_joint_create(concord_joint **out, int p, int precision, int device);
int concord_joint_destroy(concord_joint *jt);   /* NULL is accepted */
/* Stream for every later call (NULL = the state's own stream). */
int concord_joint_set_stream(concord_joint *jt, void *stream);
/* Limit of each device-side wait (default 2 s); see concord_set_timeout. */
int concord_joint_set_timeout(concord_joint *jt, double seconds);
/* CTAs of the persistent launch (0 = automatic: one warp per pair of a
 * colour, at least 16 CTAs, at most one per SM). */
int concord_joint_set_grid(concord_joint *jt, int ctas);
/* Synchronisation between colour steps (same iterates either way). */
#define CONCORD_JOINT_ROWFLAGS 0  /* default: a pair waits only for its two rows'
                                     previous-colour updates (per-row version
                                     flags, release / acquire) */
#define CONCORD_JOINT_BARRIER 1   /* one grid-wide barrier per colour step */
int concord_joint_set_variant(concord_joint *jt, int variant);
/* Failure-detection testing (CONCORD_JOINT_ROWFLAGS only): row >= 0 makes
 * that row skip publishing its version at colour step `step` of the next
 * launch (counted from the launch's first colour step over all its sweeps),
 * so the wait of the pair that reads the row next runs out at the state's
 * timeout: CONCORD_E_TIMEOUT with that row and colour step in
 * timeout_vertex / timeout_step of the result.  One-shot; row < 0 clears
 * it.  No kernel faults, traps or hangs.  Errors: CONCORD_E_ARG. */
int concord_joint_set_fault(concord_joint *jt, int row, int step);

/* Copies S of population m (0 or 1; p x p, element type s_dtype, row stride
 * lds) into the state and resets Omega_m to I (W_m = S_m).  Synchronises.
 * Errors: CONCORD_E_NONPOS_DIAG (s_ii <= 0 or S not symmetric),
 * CONCORD_E_NONFINITE, CONCORD_E_ARG. */
int concord_joint_set_S(concord_joint *jt, int m, const void *S_dev, int s_dtype, int lds);
/* Warm start: Omega_m from a device buffer (symmetric, positive diagonal);
 * W_m is rebuilt.  On a rejected Omega the state's Omega_m is reset to I. */
int concord_joint_set_omega(concord_joint *jt, int m, const void *Om_dev, int dtype, int ld);
/* Omega_m of the latest iterate into a device buffer (dtype, row stride ld). */
int concord_joint_get_omega(concord_joint *jt, int m, void *Om_dev, int dtype, int ld);

/* Exactly n_sweeps joint sweeps (FP32 under CONCORD_MIXED, FP64 otherwise),
 * no stopping rule; res receives the residual and objective after them
 * (res->lambda = lambda1).  n_sweeps = 0 only evaluates.
 * Errors: CONCORD_E_ARG (S not set, lambdas < 0), CONCORD_E_NONFINITE,
 * CONCORD_E_TIMEOUT (res->timeout_vertex = the row whose wait ran out, or
 * -1 - CTA for a grid barrier; res->timeout_step = the colour step),
 * CONCORD_E_CUDA. */
int concord_joint_sweep(concord_joint *jt, double lambda1, double lambda2, int n_sweeps,
                        concord_result *res);
/* Joint sweeps until the joint KKT residual <= tol or max_sweeps (mixed: FP32
 * phase, then FP64 polish; res->sweeps_fp32 counts the FP32 sweeps).
 * Returns CONCORD_OK or CONCORD_NOT_CONVERGED (outputs filled), or an error as
 * concord_joint_sweep. */
int concord_joint_run(concord_joint *jt, double lambda1, double lambda2, double tol,
                      int max_sweeps, concord_result *res);
/* Per-sweep rows (delta, KKT residual, objective, pairs moved) of the last
 * concord_joint_sweep / _run call: min(max_rows, rows) rows into hist_host
 * (4 doubles each); *rows receives the number recorded. */
int concord_joint_get_history(concord_joint *jt, double *hist_host, int max_rows, int *rows);

/* ------------------------------------------------- batched independent problems */
/*
 * A batch holds many independent CONCORD problems (dimensions p[b], uneven
 * allowed; data of uneven n) and solves them together: one persistent
 * cooperative launch of the sweep kernel per wave of problems whose CTAs fit
 * co-resident on the device, all problems of a wave in flight at once.  In
 * the launch every problem owns a contiguous range of CTAs (its rows,
 * mailbox ring, barrier counter and partial sums are its own), runs
 * Algorithm 1's colour steps and diagonal step (Section 3.2, 3.3; Eq. 2,
 * Eq. 3 in S units) at its own pace and walks a warm-started lambda path:
 * after a lambda meets KKT <= tol (or max_sweeps, or in MIXED precision the
 * FP32 stall rule of concord_run) it records the result, optionally adds the
 * support of its Omega into the lambda's count matrix, and continues from its
 * current iterate with the next lambda.  The problems share the launch and
 * the abort word, nothing else.  This is the batched form of the parallel
 * width the colour steps expose (Section 3.3): one problem at p = 1000 fills
 * a small part of the GPU; many together fill it.
 *
 * Memory per problem (ld = p rounded up to 32, e = 4 for MIXED, 8 for FP64):
 * S, W, Omega: 3 p ld e bytes, plus per-vertex vectors and a mailbox ring;
 * plus, when n_cap > 0, staging for one problem's data and Gram at a time.
 */
typedef struct concord_batch concord_batch;

/* n_problems >= 1 problems of dimensions p[0..n_problems) (each >= 2) on
 * `device` (-1 = current) in CONCORD_MIXED (FP32 sweeps with the FP64
 * diagonal root, KKT and objective) or CONCORD_FP64.  n_cap >= 0: most data
 * rows concord_batch_gram will be given (0: S only through
 * concord_batch_set_S).  Every Omega starts at I.
 * Errors: CONCORD_E_ARG, CONCORD_E_NOMEM, CONCORD_E_CUDA (no sm_103 device). */
int concord_batch_create(concord_batch **out, int n_problems, const int *p, int precision,
                         int n_cap, int device);
int concord_batch_destroy(concord_batch *bt);              /* NULL is accepted */
int concord_batch_set_stream(concord_batch *bt, void *stream);  /* NULL: own stream */
int concord_batch_set_timeout(concord_batch *bt, double seconds); /* device waits */

/* S of problem b from a device buffer (p_b x p_b, dtype F64 / F32, row
 * stride lds, symmetric); Omega_b <- I.  Synchronises the stream.
 * Errors: CONCORD_E_ARG (index, not symmetric), CONCORD_E_NONFINITE,
 * CONCORD_E_NONPOS_DIAG. */
int concord_batch_set_S(concord_batch *bt, int b, const void *S_dev, int s_dtype, int lds);

/* S of problem b from data: the rows rows_dev[0..n_rows) (device int32
 * indices into X; NULL: all n rows) of X (device, n x p_b, row stride ldx,
 * dtype F64 / F32), prepared by `prep` (CONCORD_PREP_*) and multiplied into
 * S = Z^T Z / n_rows -- 3xTF32 on tensor cores for MIXED, FP64 for FP64
 * (as concord_gram); Omega_b <- I.  Synchronises the stream.
 * Errors: CONCORD_E_ARG (n_rows > n_cap, ...), CONCORD_E_NONPOS_DIAG
 * (constant column), CONCORD_E_NONFINITE, CONCORD_E_CUDA. */
int concord_batch_gram(concord_batch *bt, int b, const void *X_dev, int x_dtype, int n, int ldx,
                       const int *rows_dev, int n_rows, int prep);

/* Omega_b <- I and W_b <- S_b (S kept). */
int concord_batch_reset(concord_batch *bt, int b);

/* The lambda path lambdas[0..n_lambda) (host, each >= 0) on every problem,
 * from its current iterate, each lambda until KKT <= tol or max_sweeps
 * sweeps.  MIXED: FP32 sweeps; a lambda whose FP32 sweeps stop falling by
 * 10% over 4 sweeps (the FP32 rounding floor of the maintained W, or
 * progress too slow to tell apart from it) is polished in FP64 -- W rebuilt
 * in FP64 from Omega and an FP64 copy of S, FP64 sweeps to tol within the
 * lambda's remaining sweeps, one launch for every problem that stalled --
 * and its walk resumes in FP32 from the polished iterate
 * (concord_batch_set_polish(bt, 0): a stalled lambda just ends, not
 * converged, and the walk goes on).  results (host, nullable) receives
 * n_problems x n_lambda concord_result rows (problem-major; sweeps = sweeps
 * at that lambda, status CONCORD_OK when KKT <= tol, else
 * CONCORD_NOT_CONVERGED; MIXED: sweeps_fp32 = its FP32 sweeps).
 * support_dev (device, nullable; all problems of one
 * p) gains, for every problem and lambda k, 1.0 at [k][i][j] where
 * w_ij != 0 (n_lambda x p x p floats, not cleared by the call).  When the
 * rows per warp are not set, the call first autotunes them
 * (concord_batch_autotune at the middle lambda, which resets every problem
 * to Omega = I).  Synchronises the stream.
 * Errors: CONCORD_E_ARG, CONCORD_E_OCCUPANCY, CONCORD_E_TIMEOUT, CONCORD_E_CUDA. */
int concord_batch_path(concord_batch *bt, const double *lambdas, int n_lambda, double tol,
                       int max_sweeps, concord_result *results, float *support_dev);

/* The batch's work layout: each warp of a problem owns up to `rows` rows
 * (2, 4, 8, 16 or 32; 0: autotune on the next concord_batch_path), so a
 * problem of dimension p takes ceil(p / (16 rows)) CTAs of 512 threads and
 * fewer rows per warp trade co-resident problems (waves) for row-update
 * bandwidth.  Results do not depend on it. */
int concord_batch_set_rows_per_warp(concord_batch *bt, int rows);

/* MIXED: FP64 polish of stalled lambdas in concord_batch_path (1, the
 * default) or not (0). */
int concord_batch_set_polish(concord_batch *bt, int on);

/* Times `sweeps` sweeps at `lambda` on every problem for each rows-per-warp
 * choice (32, 16, 8, 4, 2; ms_per_choice, host, nullable, receives the five
 * times in ms, -1 where a choice cannot launch), keeps the fastest, and
 * resets every problem to Omega = I.  Errors: as concord_batch_path. */
int concord_batch_autotune(concord_batch *bt, double lambda, int sweeps, double *ms_per_choice);

/* The layout of the last launch: rows per warp, the largest wave's CTAs,
 * the number of waves, and the device time of the last path (or trial). */
int concord_batch_info(concord_batch *bt, int *rows_per_warp, int *ctas, int *waves,
                       double *seconds);

/* Omega_b into a device buffer (dtype F64 / F32, row stride ldo >= p_b; for
 * MIXED and F64 the diagonal is the FP64 one).  Synchronises the stream. */
int concord_batch_get_omega(concord_batch *bt, int b, void *out_dev, int dtype, int ldo);

#ifdef __cplusplus
}
#endif
#endif /* CONCORD_GB300_H */
