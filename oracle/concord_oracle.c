/*
 * CONCORD-CD / CONCORD-PCD oracle: a plain, slow, FP64 CPU implementation of
 * what the GPU path computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Conventions
 *   - Every matrix is dense, row-major, p x p (or n x p for data), FP64.
 *   - Vertices / variables are 0-based here; the paper counts from 1.
 *   - "S units": S = Z^T Z / n for the standardized data Z.  The paper writes
 *     the method with T = X^T X; T = n S.  The penalty lambda is read on the
 *     S scale (the objective below is Eq. 1 divided by n with the penalty
 *     n*lambda); the diagonal update (Eq. 2) is the same on either scale.
 *   - No blocking, fusion or reordering beyond what the paper states: the
 *     off-diagonal update is Eq. 3 written as its two direct sums, the
 *     diagonal update is Eq. 2 with its direct sum, and the sweep follows
 *     Algorithm 1 (all colours in order, then all diagonals).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -march, no fast-math),
 * so x86-64 and aarch64 give the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Planted-mistake builds for the pin tests: compiled with -DORACLE_MUTANT=k
 * the oracle carries mistake k (see tests/test_oracle_mutants.py); the normal
 * build has ORACLE_MUTANT == 0 and every MUTANT(k) below is false. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

#define OR_OK 0
#define OR_E_ARG -1
#define OR_E_NONPOS_DIAG -2

/* ------------------------------------------------------------------------ */
/* Data preparation (Section 2.1: X is centered columnwise; the standardized  */
/* reading also scales every column to unit 1/n variance).                    */
/* ------------------------------------------------------------------------ */

/* Z[k][i] = (X[k][i] - mean_i) / sd_i with mean_i = sum_k X[k][i] / n and
 * sd_i = sqrt(sum_k (X[k][i]-mean_i)^2 / n).  If scale == 0 only centering is
 * done.  Returns OR_E_NONPOS_DIAG if a column is constant and scale != 0. */
int oracle_standardize(const double *X, int n, int p, int scale, double *Z)
{
    if (n < 1 || p < 1) return OR_E_ARG;
    for (int i = 0; i < p; ++i) {
        double mean = 0.0;
        for (int k = 0; k < n; ++k) mean += X[(size_t)k * p + i];
        mean /= n;
        double ss = 0.0;
        for (int k = 0; k < n; ++k) {
            double d = X[(size_t)k * p + i] - mean;
            ss += d * d;
        }
        double sd = sqrt(ss / (MUTANT(10) ? n - 1 : n));
        if (scale && !(sd > 0.0)) return OR_E_NONPOS_DIAG;
        for (int k = 0; k < n; ++k) {
            double d = X[(size_t)k * p + i] - mean;
            Z[(size_t)k * p + i] = scale ? d / sd : d;
        }
    }
    return OR_OK;
}

/* Row i of S = Z^T Z / n: out[j] = sum_k Z[k][i] Z[k][j] / n, k ascending. */
static void gram_row(const double *Z, int n, int p, int i, double *out)
{
    for (int j = 0; j < p; ++j) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k)
            acc += Z[(size_t)k * p + i] * Z[(size_t)k * p + j];
        out[j] = MUTANT(9) ? acc : acc / n;
    }
}

/* S = Z^T Z / n, the plain triple loop (Algorithm 1, T <- X^T X, divided by
 * n).  Both triangles are computed independently (no symmetry shortcut). */
void oracle_gram(const double *Z, int n, int p, double *S)
{
    for (int i = 0; i < p; ++i) gram_row(Z, n, p, i, S + (size_t)i * p);
}

/* Selected rows of S: out[r][j] = S[rows[r]][j], the same sums as
 * oracle_gram, for checking large p one row at a time. */
void oracle_gram_rows(const double *Z, int n, int p, const int32_t *rows, int nrows,
                      double *out)
{
    for (int r = 0; r < nrows; ++r) gram_row(Z, n, p, rows[r], out + (size_t)r * p);
}

/* ------------------------------------------------------------------------ */
/* Schedule: the circle method (Section 3.2) as Algorithm 1 runs it.         */
/* ------------------------------------------------------------------------ */

/* Fills pairs[(k * (pe/2) + q) * 2 + {0,1}] for colour k = 0..pe-2 and slot
 * q = 0..pe/2-1 with the 0-based vertices of the q-th matching pair of the
 * k-th target set, in Algorithm 1's order.  A pair that holds the extra
 * vertex p (1-based p+1, present only for odd p) is written as (-1, -1):
 * step (iii) of the circle method discards it.  Returns the number of colours
 * pe - 1, where pe = p for even p and p + 1 for odd p. */
int oracle_schedule(int p, int32_t *pairs)
{
    if (p < 2) return OR_E_ARG;
    int pe = (p % 2 == 0) ? p : p + 1;
    int *j = (int *)malloc(sizeof(int) * (size_t)(pe + 1)); /* j[1..pe], 1-based */
    if (!j) return OR_E_ARG;
    for (int m = 1; m <= pe; ++m) j[m] = m; /* (j_1, ..., j_pe) <- (1, ..., pe) */
    int half = pe / 2;
    for (int k = 0; k < pe - 1; ++k) {
        /* target set I = {(j_q, j_{pe-q+1}) : q = 1..pe/2} */
        for (int q = 1; q <= half; ++q) {
            int r = j[q], s = j[pe - q + 1];
            int32_t *slot = pairs + ((size_t)k * half + (q - 1)) * 2;
            if (r == p + 1 || s == p + 1) {
                slot[0] = -1;
                slot[1] = -1;
            } else {
                slot[0] = r - 1;
                slot[1] = s - 1;
            }
        }
        /* tmp <- j_pe, (j_3..j_pe) <- (j_2..j_{pe-1}), j_2 <- tmp */
        if (MUTANT(6)) {
            int tmp = j[2];
            for (int m = 2; m < pe; ++m) j[m] = j[m + 1];
            j[pe] = tmp;
        } else {
            int tmp = j[pe];
            for (int m = pe; m >= 3; --m) j[m] = j[m - 1];
            j[2] = tmp;
        }
    }
    free(j);
    return pe - 1;
}

/* ------------------------------------------------------------------------ */
/* Coordinate updates (Section 2.1, Eq. 2 and Eq. 3), in S units.            */
/* ------------------------------------------------------------------------ */

/* Soft_tau(x) = sign(x) (|x| - tau)_+ . */
double oracle_soft(double x, double tau)
{
    double a = fabs(x) - tau;
    if (a <= 0.0) return 0.0;
    return (x > 0.0) != MUTANT(3) ? a : -a;
}

/* Eq. 3 for the pair (i, j), i != j, from explicit inputs:
 *   omega_ij <- Soft_lambda( - sum_{u != j} omega_iu s_ju
 *                            - sum_{u != i} omega_uj s_iu ) / (s_ii + s_jj)
 * om_i[u] = omega_iu (row i), om_j[u * stride] = omega_uj (column j),
 * s_i / s_j = rows i / j of S.  Returns the new value. */
double oracle_eq3(const double *om_i, const double *om_j, size_t stride,
                  const double *s_i, const double *s_j, int p, int i, int j,
                  double lambda)
{
    double a1 = 0.0, a2 = 0.0;
    for (int u = 0; u < p; ++u)
        if (u != j || MUTANT(1)) a1 += om_i[u] * s_j[u];
    for (int u = 0; u < p; ++u)
        if (u != i) a2 += om_j[(size_t)u * stride] * (MUTANT(2) ? s_j : s_i)[u];
    double den = s_i[i] + (MUTANT(4) ? 0.0 : s_j[j]);
    return oracle_soft(-a1 - a2, lambda) / den;
}

/* Eq. 3 applied in place to the pair (i, j) of Om; the symmetric entry
 * omega_ji receives the same value.  Returns the change new - old. */
double oracle_offdiag_update(const double *S, int p, double lambda, double *Om,
                             int i, int j)
{
    double old = Om[(size_t)i * p + j];
    double nw = oracle_eq3(Om + (size_t)i * p, Om + j, (size_t)p, S + (size_t)i * p,
                           S + (size_t)j * p, p, i, j, lambda);
    Om[(size_t)i * p + j] = nw;
    Om[(size_t)j * p + i] = nw;
    return nw - old;
}

/* Eq. 2 for vertex i (divided through by n), from row i of Omega and of S:
 *   c = sum_{j != i} omega_ij s_ij,
 *   omega_ii <- (-c + sqrt(c^2 + 4 s_ii)) / (2 s_ii).
 * Returns the new value. */
double oracle_eq2(const double *om_i, const double *s_i, int p, int i)
{
    double c = 0.0;
    for (int j = 0; j < p; ++j)
        if (j != i || MUTANT(5)) c += om_i[j] * s_i[j];
    double sii = s_i[i];
    return (-c + sqrt(c * c + 4.0 * sii)) / (2.0 * sii);
}

/* Eq. 2 applied in place to vertex i of Om.  Returns the change new - old. */
double oracle_diag_update(const double *S, int p, double *Om, int i)
{
    double old = Om[(size_t)i * p + i];
    double nw = oracle_eq2(Om + (size_t)i * p, S + (size_t)i * p, p, i);
    Om[(size_t)i * p + i] = nw;
    return nw - old;
}

/* ------------------------------------------------------------------------ */
/* One outer iteration of Algorithm 1.                                        */
/* ------------------------------------------------------------------------ */

/* Runs colour steps k = k_begin..k_end-1 of the table `pairs` (as written by
 * oracle_schedule, or any permutation of pairs within a colour), serially in
 * slot order.  Returns the largest |change| seen; *n_nonzero (if not NULL) is
 * increased by the number of pairs whose change was nonzero. */
double oracle_colour_steps(const double *S, int p, double lambda, double *Om,
                           const int32_t *pairs, int half, int k_begin,
                           int k_end, long long *n_nonzero)
{
    double dmax = 0.0;
    for (int k = k_begin; k < k_end; ++k)
        for (int q = 0; q < half; ++q) {
            const int32_t *slot = pairs + ((size_t)k * half + q) * 2;
            if (slot[0] < 0) continue;
            double d = oracle_offdiag_update(S, p, lambda, Om, slot[0], slot[1]);
            if (fabs(d) > dmax) dmax = fabs(d);
            if (n_nonzero && d != 0.0) ++*n_nonzero;
        }
    return dmax;
}

/* The diagonal step of Algorithm 1 for all i.  Returns the largest |change|. */
double oracle_diag_step(const double *S, int p, double *Om)
{
    double dmax = 0.0;
    for (int i = 0; i < p; ++i) {
        double d = oracle_diag_update(S, p, Om, i);
        if (fabs(d) > dmax) dmax = fabs(d);
    }
    return dmax;
}

/* One full sweep: all n_colours colour steps in order, then the diagonal
 * step.  Returns delta = |Omega^(t) - Omega^(t-1)|_inf.  Every entry is
 * written once per sweep, so the largest single change is that norm. */
double oracle_sweep(const double *S, int p, double lambda, double *Om,
                    const int32_t *pairs, int n_colours, long long *n_nonzero)
{
    int half = (n_colours + 1) / 2;
    double d1 = oracle_colour_steps(S, p, lambda, Om, pairs, half, 0, n_colours,
                                    n_nonzero);
    double d2 = oracle_diag_step(S, p, Om);
    return d1 > d2 ? d1 : d2;
}

/* ------------------------------------------------------------------------ */
/* Objective (Eq. 1) and optimality.                                          */
/* ------------------------------------------------------------------------ */

/* Eq. 1 divided by n, from S:
 *   f = - sum_i log omega_ii + 1/2 sum_i (Omega S Omega)_ii
 *       + lambda sum_{i<j} |omega_ij|.
 * (Omega S Omega)_ii is formed as the double sum over a, b of
 * omega_ia s_ab omega_bi.  Returns NaN if a diagonal entry is not positive. */
double oracle_objective(const double *S, const double *Om, int p, double lambda)
{
    double logs = 0.0, quad = 0.0, pen = 0.0;
    for (int i = 0; i < p; ++i) {
        double w = Om[(size_t)i * p + i];
        if (!(w > 0.0)) return NAN;
        logs += log(w);
    }
    for (int i = 0; i < p; ++i) {
        double acc = 0.0;
        for (int a = 0; a < p; ++a) {
            double oia = Om[(size_t)i * p + a];
            if (oia == 0.0) continue;
            double inner = 0.0;
            for (int b = 0; b < p; ++b)
                inner += S[(size_t)a * p + b] * Om[(size_t)b * p + i];
            acc += oia * inner;
        }
        quad += acc;
    }
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) pen += fabs(Om[(size_t)i * p + j]);
    return -logs + (MUTANT(8) ? 1.0 : 0.5) * quad + lambda * pen;
}

/* Eq. 1 divided by n, from the (centered / standardized) data Z directly:
 *   f = - sum_i log omega_ii
 *       + 1/(2n) sum_i sum_k (omega_ii Z_ki + sum_{j != i} omega_ij Z_kj)^2
 *       + lambda sum_{i<j} |omega_ij|. */
double oracle_objective_data(const double *Z, int n, const double *Om, int p,
                             double lambda)
{
    double logs = 0.0, quad = 0.0, pen = 0.0;
    for (int i = 0; i < p; ++i) {
        double w = Om[(size_t)i * p + i];
        if (!(w > 0.0)) return NAN;
        logs += log(w);
    }
    for (int i = 0; i < p; ++i)
        for (int k = 0; k < n; ++k) {
            double r = Om[(size_t)i * p + i] * Z[(size_t)k * p + i];
            for (int j = 0; j < p; ++j)
                if (j != i) r += Om[(size_t)i * p + j] * Z[(size_t)k * p + j];
            quad += r * r;
        }
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) pen += fabs(Om[(size_t)i * p + j]);
    return -logs + quad / (2.0 * n) + lambda * pen;
}

/* Largest violation of the subgradient optimality conditions of f (absolute,
 * S units).  With W = Omega S and G = W + W^T (the gradient of the smooth
 * part with respect to the shared variable omega_ij = omega_ji):
 *   diagonal i:             | W_ii - 1/omega_ii |
 *   off-diagonal, w != 0:   | G_ij + lambda sign(omega_ij) |
 *   off-diagonal, w == 0:   max(|G_ij| - lambda, 0).
 * W is formed here by the plain product. */
double oracle_kkt(const double *S, const double *Om, int p, double lambda)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)p * p);
    if (!W) return NAN;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            double acc = 0.0;
            for (int u = 0; u < p; ++u) {
                double o = Om[(size_t)i * p + u];
                if (o != 0.0) acc += o * S[(size_t)u * p + j]; /* exact zeros add nothing */
            }
            W[(size_t)i * p + j] = acc;
        }
    double worst = 0.0;
    for (int i = 0; i < p; ++i) {
        double wii = Om[(size_t)i * p + i];
        double r = (wii > 0.0) ? fabs(W[(size_t)i * p + i] - 1.0 / wii) : INFINITY;
        if (r > worst) worst = r;
        for (int j = i + 1; j < p; ++j) {
            double g = W[(size_t)i * p + j] + W[(size_t)j * p + i];
            double w = Om[(size_t)i * p + j];
            double v;
            if (w > 0.0)
                v = fabs(MUTANT(7) ? g - lambda : g + lambda);
            else if (w < 0.0)
                v = fabs(MUTANT(7) ? g + lambda : g - lambda);
            else
                v = fabs(g) - lambda > 0.0 ? fabs(g) - lambda : 0.0;
            if (v > worst) worst = v;
        }
    }
    free(W);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Driver: Algorithm 1 repeated until the stopping rule holds.               */
/* ------------------------------------------------------------------------ */

/* stats layout (doubles), written on return:
 *   [0] sweeps done   [1] objective   [2] KKT residual   [3] last delta
 *   [4] first sweep at which delta < delta_tol (0 if never)
 *   [5] nonzero pair changes in the last sweep
 * Stops when KKT <= tol (checked after every sweep) or at max_sweeps.
 * Om0 may be NULL (start from the identity).  history, if not NULL, receives
 * (delta, kkt, objective) for every sweep (3 * max_sweeps doubles).
 * Returns 0 if converged, 1 if not, <0 on argument errors. */
int oracle_solve(const double *S, int p, double lambda, double tol,
                 double delta_tol, int max_sweeps, const double *Om0,
                 double *Om, double *stats, double *history)
{
    if (p < 2 || !(lambda >= 0.0) || !(tol > 0.0) || max_sweeps < 0) return OR_E_ARG;
    for (int i = 0; i < p; ++i)
        if (!(S[(size_t)i * p + i] > 0.0)) return OR_E_NONPOS_DIAG;
    int pe = (p % 2 == 0) ? p : p + 1;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pe - 1) * (pe / 2) * 2);
    if (!pairs) return OR_E_ARG;
    int nc = oracle_schedule(p, pairs);
    if (Om0)
        memcpy(Om, Om0, sizeof(double) * (size_t)p * p);
    else
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) Om[(size_t)i * p + j] = (i == j) ? 1.0 : 0.0;
    int t = 0, first_delta = 0, status = 1;
    double delta = 0.0, kkt = oracle_kkt(S, Om, p, lambda);
    long long nnz = 0;
    while (t < max_sweeps) {
        nnz = 0;
        delta = oracle_sweep(S, p, lambda, Om, pairs, nc, &nnz);
        ++t;
        kkt = oracle_kkt(S, Om, p, lambda);
        if (history) {
            history[3 * (t - 1) + 0] = delta;
            history[3 * (t - 1) + 1] = kkt;
            history[3 * (t - 1) + 2] = oracle_objective(S, Om, p, lambda);
        }
        if (!first_delta && delta < delta_tol) first_delta = t;
        if (kkt <= tol) {
            status = 0;
            break;
        }
    }
    if (max_sweeps == 0 && kkt <= tol) status = 0;
    stats[0] = t;
    stats[1] = oracle_objective(S, Om, p, lambda);
    stats[2] = kkt;
    stats[3] = delta;
    stats[4] = first_delta;
    stats[5] = (double)nnz;
    free(pairs);
    return status;
}
