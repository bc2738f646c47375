/*
 * CONCORD-PCD oracle, maintained-product mode: the timed CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY, like concord_oracle.c (the definition mode) in
 * this folder: only the tests, the smoke check and the benchmark's CPU legs
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * What it computes: exactly what oracle_solve computes (Algorithm 1 in the
 * colour order of the circle method, then the diagonal step, until the KKT
 * residual meets tol), in S units, FP64.  Two things differ, both stated by
 * the paper:
 *
 *   - The sums of Eq. 3 and Eq. 2 are read off a maintained product
 *     W = Omega S instead of being summed directly.  Row i of W is
 *     sum_u omega_iu S_u, so
 *        sum_{u != j} omega_iu s_ju = W_ij - omega_ij s_jj,
 *        sum_{u != i} omega_uj s_iu = W_ji - omega_ij s_ii   (symmetry),
 *        sum_{j != i} omega_ij s_ij = W_ii - omega_ii s_ii,
 *     and a change d of omega_ij = omega_ji adds d S_j to row i and d S_i to
 *     row j of W; a change of omega_ii adds it times S_i to row i.
 *   - The pairs of one colour are spread over OpenMP threads (Lemma 1: they
 *     read and write disjoint rows of Omega and W), and so are the p
 *     diagonal updates (Algorithm 1 updates them "in parallel": the update of
 *     vertex i reads and writes only row i).  This is the paper's PCD run on
 *     the host cores (its PCD-CPU comparison, Section 5).
 *
 * Results do not depend on the thread count: every entry is computed by one
 * thread with a fixed order of operations, and every sum over rows is formed
 * per row and then added up serially.  They differ from the definition mode
 * only by rounding order (the maintained W accumulates its updates), which
 * the tests bound at p <= 1000.
 *
 * Build: with concord_oracle.c, gcc -O2 -ffp-contract=off -fopenmp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_schedule(int p, int32_t *pairs);
double oracle_soft(double x, double tau);

/* Planted-mistake builds (tests/test_oracle_mutants.py): -DORACLE_MUTANT=k
 * with k = 15..17 puts mistake k into this file; 0 is the normal build. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

#define ORW_E_ARG -1
#define ORW_E_NONPOS_DIAG -2

static int set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* Threads this build runs with for a request of `threads` (0 = all). */
int oracle_w_threads(int threads)
{
    return set_threads(threads);
}

/* S = Z^T Z / n (Algorithm 1, T <- X^T X, divided by n), upper triangle
 * computed with k ascending and mirrored.  Rows of the result are spread over
 * the threads; Z is read through its transpose so the sums walk contiguous
 * memory. */
int oracle_w_gram(const double *Z, int n, int p, double *S, int threads)
{
    if (n < 1 || p < 1) return ORW_E_ARG;
    set_threads(threads);
    double *Zt = (double *)malloc(sizeof(double) * (size_t)n * p);
    if (!Zt) return ORW_E_ARG;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p; ++i)
        for (int k = 0; k < n; ++k) Zt[(size_t)i * n + k] = Z[(size_t)k * p + i];
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < p; ++i) {
        const double *zi = Zt + (size_t)i * n;
        for (int j = i; j < p; ++j) {
            const double *zj = Zt + (size_t)j * n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += zi[k] * zj[k];
            S[(size_t)i * p + j] = acc / n;
        }
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < i; ++j) S[(size_t)i * p + j] = S[(size_t)j * p + i];
    free(Zt);
    return 0;
}

/* W = Omega S, rows over threads, u ascending, exact zeros of Omega skipped. */
static void product(const double *S, const double *Om, int p, double *W)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p; ++i) {
        double *w = W + (size_t)i * p;
        for (int j = 0; j < p; ++j) w[j] = 0.0;
        for (int u = 0; u < p; ++u) {
            double o = Om[(size_t)i * p + u];
            if (o == 0.0) continue;
            const double *s = S + (size_t)u * p;
            for (int j = 0; j < p; ++j) w[j] += o * s[j];
        }
    }
}

/* Row i of W gains d times row u of S. */
static void row_axpy(double *W, const double *S, int p, int i, int u, double d)
{
    double *w = W + (size_t)i * p;
    const double *s = S + (size_t)u * p;
    for (int j = 0; j < p; ++j) w[j] += d * s[j];
}

/* KKT residual (the definition of oracle_kkt) and objective (Eq. 1 / n) from
 * the maintained W; per-row parts, added serially. */
static void kkt_objective(const double *S, const double *Om, const double *W, int p,
                          double lambda, double *row_a, double *row_b, double *row_c,
                          double *kkt, double *obj)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < p; ++i) {
        const double *w = W + (size_t)i * p;
        const double *o = Om + (size_t)i * p;
        double wii = o[i];
        double worst = (wii > 0.0) ? fabs(w[i] - 1.0 / wii) : INFINITY;
        double quad = 0.0, pen = 0.0;
        for (int j = 0; j < p; ++j) quad += w[j] * o[j]; /* (W Omega)_ii, Omega symmetric */
        for (int j = i + 1; j < p; ++j) {
            double g = w[j] + W[(size_t)j * p + i];
            double om = o[j];
            double v;
            if (om > 0.0)
                v = fabs(g + lambda);
            else if (om < 0.0)
                v = fabs(g - lambda);
            else
                v = fabs(g) - lambda > 0.0 ? fabs(g) - lambda : 0.0;
            if (v > worst) worst = v;
            pen += fabs(om);
        }
        row_a[i] = worst;
        row_b[i] = quad;
        row_c[i] = pen;
    }
    double worst = 0.0, logs = 0.0, quad = 0.0, pen = 0.0;
    for (int i = 0; i < p; ++i) {
        double wii = Om[(size_t)i * p + i];
        if (row_a[i] > worst || isnan(row_a[i])) worst = row_a[i];
        logs += (wii > 0.0) ? log(wii) : NAN;
        quad += row_b[i];
        pen += row_c[i];
    }
    (void)S;
    *kkt = worst;
    *obj = -logs + 0.5 * quad + lambda * pen;
}

/* The solve of oracle_solve with a maintained W and threads: the same
 * arguments, stats layout and history layout (delta, kkt, objective per
 * sweep), plus `threads` (0 = all host cores).  stats[6] receives the thread
 * count used. */
int oracle_solve_w(const double *S, int p, double lambda, double tol, double delta_tol,
                   int max_sweeps, const double *Om0, double *Om, double *stats,
                   double *history, int threads)
{
    if (p < 2 || !(lambda >= 0.0) || !(tol > 0.0) || max_sweeps < 0) return ORW_E_ARG;
    for (int i = 0; i < p; ++i)
        if (!(S[(size_t)i * p + i] > 0.0)) return ORW_E_NONPOS_DIAG;
    int used = set_threads(threads);
    int pe = (p % 2 == 0) ? p : p + 1;
    int half = pe / 2;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pe - 1) * half * 2);
    double *W = (double *)malloc(sizeof(double) * (size_t)p * p);
    double *scratch = (double *)malloc(sizeof(double) * (size_t)(3 * p + half));
    if (!pairs || !W || !scratch) {
        free(pairs);
        free(W);
        free(scratch);
        return ORW_E_ARG;
    }
    double *row_a = scratch, *row_b = scratch + p, *row_c = scratch + 2 * p;
    double *pair_d = scratch + 3 * p;
    int n_colours = oracle_schedule(p, pairs);
    if (Om0)
        memcpy(Om, Om0, sizeof(double) * (size_t)p * p);
    else
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) Om[(size_t)i * p + j] = (i == j) ? 1.0 : 0.0;
    product(S, Om, p, W);
    double kkt, obj;
    kkt_objective(S, Om, W, p, lambda, row_a, row_b, row_c, &kkt, &obj);
    int t = 0, first_delta = 0, status = 1;
    double delta = 0.0;
    long long nnz = 0;
    while (t < max_sweeps) {
        nnz = 0;
        delta = 0.0;
        for (int k = 0; k < n_colours; ++k) {
            const int32_t *colour = pairs + (size_t)k * half * 2;
            /* Eq. 3 for every pair of colour k at once (Lemma 1) */
#pragma omp parallel for schedule(static)
            for (int q = 0; q < half; ++q) {
                int i = colour[2 * q], j = colour[2 * q + 1];
                pair_d[q] = 0.0;
                if (i < 0) continue;
                double sii = S[(size_t)i * p + i], sjj = S[(size_t)j * p + j];
                double old = Om[(size_t)i * p + j];
                double a1 = W[(size_t)i * p + j] - (MUTANT(15) ? 0.0 : old * sjj); /* sum_{u != j} omega_iu s_ju */
                double a2 = W[(size_t)j * p + i] - old * sii; /* sum_{u != i} omega_uj s_iu */
                double nw = oracle_soft(-a1 - a2, lambda) / (sii + sjj);
                double d = nw - old;
                pair_d[q] = d;
                if (d == 0.0) continue;
                Om[(size_t)i * p + j] = nw;
                Om[(size_t)j * p + i] = nw;
                row_axpy(W, S, p, i, j, d);
                if (!MUTANT(16)) row_axpy(W, S, p, j, i, d);
            }
            for (int q = 0; q < half; ++q) {
                double d = fabs(pair_d[q]);
                if (d > delta) delta = d;
                if (pair_d[q] != 0.0) ++nnz;
            }
        }
        /* Eq. 2 for every vertex at once */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < p; ++i) {
            double sii = S[(size_t)i * p + i];
            double old = Om[(size_t)i * p + i];
            double c = W[(size_t)i * p + i] - old * sii; /* sum_{j != i} omega_ij s_ij */
            double nw = (-c + sqrt(c * c + 4.0 * sii)) / (2.0 * sii);
            double d = nw - old;
            row_a[i] = d;
            if (d == 0.0) continue;
            Om[(size_t)i * p + i] = nw;
            if (!MUTANT(17)) row_axpy(W, S, p, i, i, d);
        }
        for (int i = 0; i < p; ++i)
            if (fabs(row_a[i]) > delta) delta = fabs(row_a[i]);
        ++t;
        kkt_objective(S, Om, W, p, lambda, row_a, row_b, row_c, &kkt, &obj);
        if (history) {
            history[3 * (t - 1) + 0] = delta;
            history[3 * (t - 1) + 1] = kkt;
            history[3 * (t - 1) + 2] = obj;
        }
        if (!first_delta && delta < delta_tol) first_delta = t;
        if (kkt <= tol) {
            status = 0;
            break;
        }
    }
    if (max_sweeps == 0 && kkt <= tol) status = 0;
    stats[0] = t;
    stats[1] = obj;
    stats[2] = kkt;
    stats[3] = delta;
    stats[4] = first_delta;
    stats[5] = (double)nnz;
    stats[6] = used;
    free(pairs);
    free(W);
    free(scratch);
    return status;
}
