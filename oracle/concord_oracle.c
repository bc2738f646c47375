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
/* Schedule: the circle method of Section 3.2.                               */
/* ------------------------------------------------------------------------ */

/* The round-robin table of Section 3.2, step (i), has two rows of pe/2
 * cells.  Vertex 1 stays in the top-left cell; the other m = pe - 1 vertices
 * sit on a circle that runs left to right along the top row (columns
 * 2..pe/2) and then right to left along the bottom row (columns pe/2..1).
 * Counting circle positions from 0 at the top of column 2, the top cell of
 * column t >= 2 is position t - 2 and the bottom cell of column t >= 1 is
 * position pe - 1 - t.  The first table fills the circle with 2, 3, ..., pe
 * in that order, and every later table turns it one position clockwise, so
 * in table k (1-based) position c holds the vertex that was at position
 * c - (k - 1) in the first table. */
static int circle_vertex(int c, int k, int pe)
{
    int m = pe - 1;
    int shift = MUTANT(6) ? -(k - 1) : (k - 1); /* mutant: turned the wrong way */
    int r = ((c - shift) % m + m) % m;
    return 2 + r; /* 1-based vertex */
}

/* Fills pairs[(k * (pe/2) + q) * 2 + {0,1}] for colour k = 0..pe-2 and column
 * q = 0..pe/2-1 with the 0-based (top, bottom) vertices of column q + 1 of
 * table k + 1: step (ii) takes the two vertices of a column as a matching
 * pair and the k-th table's columns as the k-th target set, step (iv) gives
 * that set the k-th colour (Algorithm 1 visits the colours in this order).
 * A column holding the extra vertex p + 1 (odd p only) is written as
 * (-1, -1): step (iii) discards it.  Returns the number of colours pe - 1,
 * with pe = p for even p and p + 1 for odd p. */
int oracle_schedule(int p, int32_t *pairs)
{
    if (p < 2) return OR_E_ARG;
    int pe = (p % 2 == 0) ? p : p + 1;
    int half = pe / 2;
    for (int k = 1; k <= pe - 1; ++k) {
        for (int t = 1; t <= half; ++t) {
            int top = (t == 1) ? 1 : circle_vertex(t - 2, k, pe);
            int bottom = circle_vertex(pe - 1 - t, k, pe);
            int32_t *slot = pairs + ((size_t)(k - 1) * half + (t - 1)) * 2;
            if (top == p + 1 || bottom == p + 1) {
                slot[0] = -1;
                slot[1] = -1;
            } else {
                slot[0] = top - 1;
                slot[1] = bottom - 1;
            }
        }
    }
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
/* The two direct sums of Eq. 3: a1 = sum_{u != j} omega_iu s_ju and
 * a2 = sum_{u != i} omega_uj s_iu. */
static void eq3_sums(const double *om_i, const double *om_j, size_t stride,
                     const double *s_i, const double *s_j, int p, int i, int j,
                     double *a1_out, double *a2_out)
{
    double a1 = 0.0, a2 = 0.0;
    for (int u = 0; u < p; ++u)
        if (u != j || MUTANT(1)) a1 += om_i[u] * s_j[u];
    for (int u = 0; u < p; ++u)
        if (u != i) a2 += om_j[(size_t)u * stride] * (MUTANT(2) ? s_j : s_i)[u];
    *a1_out = a1;
    *a2_out = a2;
}

double oracle_eq3(const double *om_i, const double *om_j, size_t stride,
                  const double *s_i, const double *s_j, int p, int i, int j,
                  double lambda)
{
    double a1, a2;
    eq3_sums(om_i, om_j, stride, s_i, s_j, p, i, j, &a1, &a2);
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
/* The direct sum of Eq. 2: c = sum_{j != i} omega_ij s_ij. */
static double eq2_sum(const double *om_i, const double *s_i, int p, int i)
{
    double c = 0.0;
    for (int j = 0; j < p; ++j)
        if (j != i || MUTANT(5)) c += om_i[j] * s_i[j];
    return c;
}

double oracle_eq2(const double *om_i, const double *s_i, int p, int i)
{
    double c = eq2_sum(om_i, s_i, p, i);
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
    /* W_ij = sum_u omega_iu s_uj with u ascending for every j; exact zeros of
     * Omega add nothing and are skipped, so a row costs nnz(row) * p. */
    for (int i = 0; i < p; ++i) {
        double *w = W + (size_t)i * p;
        for (int j = 0; j < p; ++j) w[j] = 0.0;
        for (int u = 0; u < p; ++u) {
            double o = Om[(size_t)i * p + u];
            if (o == 0.0) continue;
            for (int j = 0; j < p; ++j) w[j] += o * S[(size_t)u * p + j];
        }
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

/* ======================================================================== */
/* Joint two-population CONCORD (the extension at the end of Section 6).     */
/* ======================================================================== */
/*
 * Two precision matrices Omega1, Omega2 (one per population, Grams S1, S2 in
 * S units) minimise the sum of the two populations' Eq. 1 objectives with
 * the lasso weight lambda1 on every off-diagonal entry of each matrix, plus
 * the fusion penalty lambda2 sum_{i <= j} |omega1_ij - omega2_ij| (the
 * diagonal included, as the joint objective writes it).  With a common n the
 * joint objective divided by n is exactly this; penalties are on the S scale.
 *
 * Block coordinate descent moves the pair (omega1_ij, omega2_ij) jointly, in
 * the colour order of Algorithm 1 (disjoint pairs do not interact, the same
 * argument as Lemma 1), then the diagonal blocks (omega1_ii, omega2_ii).
 */

/* Minimiser of the strictly convex two-variable block problem
 *   q(x, y) = c1 x^2 / 2 + g1 x + c2 y^2 / 2 + g2 y
 *             + l1 (|x| + |y|) + l2 |x - y|,        c1, c2 > 0.
 * If the minimiser has x > y, |x - y| = x - y near it and q separates into
 * two lasso problems: x = Soft_l1(-(g1 + l2)) / c1, y = Soft_l1(-(g2 - l2)) / c2;
 * conversely, if those values satisfy x > y they meet every subgradient
 * condition of q and are its minimiser.  The same holds with the signs of l2
 * swapped for x < y.  Otherwise x = y = t with t the minimiser of q on the
 * line x = y: t = Soft_{2 l1}(-(g1 + g2)) / (c1 + c2).  Exactly one of the
 * three cases holds in exact arithmetic. */
void oracle_joint_pair(double c1, double g1, double c2, double g2, double l1,
                       double l2, double *x, double *y)
{
    double xa = oracle_soft(-(g1 + l2), l1) / c1;
    double ya = oracle_soft(-(g2 - (MUTANT(11) ? -l2 : l2)), l1) / c2;
    if (xa > ya) {
        *x = xa;
        *y = ya;
        return;
    }
    double xb = oracle_soft(-(g1 - l2), l1) / c1;
    double yb = oracle_soft(-(g2 + l2), l1) / c2;
    if (xb < yb) {
        *x = xb;
        *y = yb;
        return;
    }
    double t = oracle_soft(-(g1 + g2), 2.0 * l1) / (c1 + c2);
    *x = t;
    *y = t;
}

/* Positive root of s d^2 + b d - 1 = 0, i.e. of -1/d + s d + b = 0 (the
 * stationarity condition Eq. 2 solves). */
static double joint_root(double s, double b)
{
    return (-b + sqrt(b * b + 4.0 * s)) / (2.0 * s);
}

/* Minimiser over d1, d2 > 0 of the diagonal block problem
 *   -log d1 + s1 d1^2 / 2 + b1 d1 - log d2 + s2 d2^2 / 2 + b2 d2 + l2 |d1 - d2|.
 * The same three cases as oracle_joint_pair: d1 > d2 gives the two Eq. 2
 * roots with b1 + l2 and b2 - l2; d1 < d2 the roots with b1 - l2 and b2 + l2;
 * otherwise d1 = d2 = d, the positive root of
 * (s1 + s2) d^2 + (b1 + b2) d - 2 = 0. */
void oracle_joint_diag(double s1, double b1, double s2, double b2, double l2,
                       double *d1, double *d2)
{
    double ua = joint_root(s1, b1 + l2), va = joint_root(s2, b2 - l2);
    if (ua > va) {
        *d1 = ua;
        *d2 = va;
        return;
    }
    double ub = joint_root(s1, b1 - l2), vb = joint_root(s2, b2 + l2);
    if (ub < vb) {
        *d1 = ub;
        *d2 = vb;
        return;
    }
    double ss = s1 + s2, bb = b1 + b2;
    double d = (-bb + sqrt(bb * bb + (MUTANT(12) ? 4.0 : 8.0) * ss)) / (2.0 * ss);
    *d1 = d;
    *d2 = d;
}

/* The joint update of the pair (i, j): for population m the direct sums of
 * Eq. 3 give g_m = sum_{u != j} omega^m_iu s^m_ju + sum_{u != i} omega^m_uj s^m_iu
 * and c_m = s^m_ii + s^m_jj; the block minimiser is written to both triangles
 * of both matrices.  Returns the larger |change|. */
double oracle_joint_offdiag_update(const double *S1, const double *S2, int p,
                                   double l1, double l2, double *Om1,
                                   double *Om2, int i, int j)
{
    const double *S[2] = {S1, S2};
    double *Om[2] = {Om1, Om2};
    double g[2], c[2], old[2];
    for (int m = 0; m < 2; ++m) {
        double a1, a2;
        eq3_sums(Om[m] + (size_t)i * p, Om[m] + j, (size_t)p, S[m] + (size_t)i * p,
                 S[m] + (size_t)j * p, p, i, j, &a1, &a2);
        g[m] = a1 + a2;
        c[m] = S[m][(size_t)i * p + i] + S[m][(size_t)j * p + j];
        old[m] = Om[m][(size_t)i * p + j];
    }
    double nw[2];
    oracle_joint_pair(c[0], g[0], c[1], g[1], l1, l2, &nw[0], &nw[1]);
    double dmax = 0.0;
    for (int m = 0; m < 2; ++m) {
        Om[m][(size_t)i * p + j] = nw[m];
        Om[m][(size_t)j * p + i] = nw[m];
        double d = fabs(nw[m] - old[m]);
        if (d > dmax) dmax = d;
    }
    return dmax;
}

/* The joint diagonal update of vertex i: b_m is the direct sum of Eq. 2 for
 * population m.  Returns the larger |change|. */
double oracle_joint_diag_update(const double *S1, const double *S2, int p,
                                double l2, double *Om1, double *Om2, int i)
{
    size_t ii = (size_t)i * p + i;
    double b1 = eq2_sum(Om1 + (size_t)i * p, S1 + (size_t)i * p, p, i);
    double b2 = eq2_sum(Om2 + (size_t)i * p, S2 + (size_t)i * p, p, i);
    double d1, d2;
    oracle_joint_diag(S1[ii], b1, S2[ii], b2, l2, &d1, &d2);
    double c1 = fabs(d1 - Om1[ii]), c2 = fabs(d2 - Om2[ii]);
    Om1[ii] = d1;
    Om2[ii] = d2;
    return c1 > c2 ? c1 : c2;
}

/* One joint sweep: every colour of `pairs` in order (slot order within a
 * colour), then every diagonal block.  Returns the largest |change| of any
 * entry of either matrix; *n_nonzero counts the pairs that moved. */
double oracle_joint_sweep(const double *S1, const double *S2, int p, double l1,
                          double l2, double *Om1, double *Om2,
                          const int32_t *pairs, int n_colours, long long *n_nonzero)
{
    int half = (n_colours + 1) / 2;
    double dmax = 0.0;
    for (int k = 0; k < n_colours; ++k)
        for (int q = 0; q < half; ++q) {
            const int32_t *slot = pairs + ((size_t)k * half + q) * 2;
            if (slot[0] < 0) continue;
            double d = oracle_joint_offdiag_update(S1, S2, p, l1, l2, Om1, Om2,
                                                   slot[0], slot[1]);
            if (d > dmax) dmax = d;
            if (n_nonzero && d != 0.0) ++*n_nonzero;
        }
    for (int i = 0; i < p; ++i) {
        double d = oracle_joint_diag_update(S1, S2, p, l2, Om1, Om2, i);
        if (d > dmax) dmax = d;
    }
    return dmax;
}

/* Joint objective (S units): the two populations' Eq. 1 objectives with
 * lasso weight l1, plus l2 sum_{i <= j} |omega1_ij - omega2_ij|. */
double oracle_joint_objective(const double *S1, const double *S2, const double *Om1,
                              const double *Om2, int p, double l1, double l2)
{
    double f = oracle_objective(S1, Om1, p, l1) + oracle_objective(S2, Om2, p, l1);
    double fus = 0.0;
    for (int i = 0; i < p; ++i)
        for (int j = (MUTANT(13) ? i + 1 : i); j < p; ++j)
            fus += fabs(Om1[(size_t)i * p + j] - Om2[(size_t)i * p + j]);
    return f + l2 * fus;
}

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Distance from -g to the set l1 * d|x| (the lasso subdifferential). */
static double lasso_residual(double g, double x, double l1)
{
    if (x > 0.0) return fabs(g + l1);
    if (x < 0.0) return fabs(g - l1);
    double r = fabs(g) - l1;
    return r > 0.0 ? r : 0.0;
}

/* Largest violation of the subgradient optimality conditions of the joint
 * objective (absolute, S units).  W_m = Omega_m S_m by the plain product.
 * For a pair (i < j) with smooth gradients G_m = W^m_ij + W^m_ji, the
 * conditions ask for u = l2 z, z in d|x - y|, with
 *   0 in G1 + u + l1 d|x|   and   0 in G2 - u + l1 d|y|;
 * the residual is the smallest, over admissible u, of the larger of the two
 * distances.  If x != y, u = l2 sign(x - y) is fixed.  If x = y both
 * distances are |A + u| and |B - u| (A, B the gradients with the lasso term
 * of a nonzero x folded in; for x = y = 0 the distances are those minus l1,
 * floored at 0), whose maximum is convex in u and smallest at
 * u = (B - A) / 2, so the admissible optimum is that u clamped to
 * [-l2, l2].  Diagonal blocks: G_m = W^m_ii - 1 / omega^m_ii, no lasso term,
 * the same rule for u. */
double oracle_joint_kkt(const double *S1, const double *S2, const double *Om1,
                        const double *Om2, int p, double l1, double l2)
{
    const double *S[2] = {S1, S2};
    const double *Om[2] = {Om1, Om2};
    double *W[2];
    for (int m = 0; m < 2; ++m) {
        W[m] = (double *)malloc(sizeof(double) * (size_t)p * p);
        if (!W[m]) {
            if (m) free(W[0]);
            return NAN;
        }
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int u = 0; u < p; ++u) {
                    double o = Om[m][(size_t)i * p + u];
                    if (o != 0.0) acc += o * S[m][(size_t)u * p + j];
                }
                W[m][(size_t)i * p + j] = acc;
            }
    }
    double worst = 0.0;
    for (int i = 0; i < p; ++i) {
        size_t ii = (size_t)i * p + i;
        double d1 = Om1[ii], d2 = Om2[ii];
        double r;
        if (!(d1 > 0.0) || !(d2 > 0.0)) {
            r = INFINITY;
        } else {
            double a = W[0][ii] - 1.0 / d1, b = W[1][ii] - 1.0 / d2;
            double u;
            if (d1 != d2)
                u = d1 > d2 ? l2 : -l2;
            else
                u = MUTANT(14) ? 0.0 : clampd(0.5 * (b - a), -l2, l2);
            double ra = fabs(a + u), rb = fabs(b - u);
            r = ra > rb ? ra : rb;
        }
        if (r > worst) worst = r;
        for (int j = i + 1; j < p; ++j) {
            size_t ij = (size_t)i * p + j, ji = (size_t)j * p + i;
            double x = Om1[ij], y = Om2[ij];
            double g1 = W[0][ij] + W[0][ji], g2 = W[1][ij] + W[1][ji];
            double v;
            if (x != y) {
                double u = x > y ? l2 : -l2;
                double r1 = lasso_residual(g1 + u, x, l1), r2 = lasso_residual(g2 - u, y, l1);
                v = r1 > r2 ? r1 : r2;
            } else if (x != 0.0) {
                double sg = x > 0.0 ? l1 : -l1;
                double A = g1 + sg, B = g2 + sg;
                double u = MUTANT(14) ? 0.0 : clampd(0.5 * (B - A), -l2, l2);
                double ra = fabs(A + u), rb = fabs(B - u);
                v = ra > rb ? ra : rb;
            } else {
                double u = MUTANT(14) ? 0.0 : clampd(0.5 * (g2 - g1), -l2, l2);
                double ra = fabs(g1 + u), rb = fabs(g2 - u);
                double m = (ra > rb ? ra : rb) - l1;
                v = m > 0.0 ? m : 0.0;
            }
            if (v > worst) worst = v;
        }
    }
    free(W[0]);
    free(W[1]);
    return worst;
}

/* Joint driver: joint sweeps until the joint KKT residual <= tol or
 * max_sweeps.  stats / history as oracle_solve (history rows: delta, KKT,
 * joint objective).  Om0_1 / Om0_2 may be NULL (identity).  Returns 0 if
 * converged, 1 if not, < 0 on argument errors. */
int oracle_joint_solve(const double *S1, const double *S2, int p, double l1,
                       double l2, double tol, double delta_tol, int max_sweeps,
                       const double *Om0_1, const double *Om0_2, double *Om1,
                       double *Om2, double *stats, double *history)
{
    if (p < 2 || !(l1 >= 0.0) || !(l2 >= 0.0) || !(tol > 0.0) || max_sweeps < 0)
        return OR_E_ARG;
    for (int i = 0; i < p; ++i)
        if (!(S1[(size_t)i * p + i] > 0.0) || !(S2[(size_t)i * p + i] > 0.0))
            return OR_E_NONPOS_DIAG;
    int pe = (p % 2 == 0) ? p : p + 1;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pe - 1) * (pe / 2) * 2);
    if (!pairs) return OR_E_ARG;
    int nc = oracle_schedule(p, pairs);
    const double *init[2] = {Om0_1, Om0_2};
    double *Om[2] = {Om1, Om2};
    for (int m = 0; m < 2; ++m) {
        if (init[m])
            memcpy(Om[m], init[m], sizeof(double) * (size_t)p * p);
        else
            for (int i = 0; i < p; ++i)
                for (int j = 0; j < p; ++j) Om[m][(size_t)i * p + j] = (i == j) ? 1.0 : 0.0;
    }
    int t = 0, first_delta = 0, status = 1;
    double delta = 0.0, kkt = oracle_joint_kkt(S1, S2, Om1, Om2, p, l1, l2);
    long long nnz = 0;
    while (t < max_sweeps) {
        nnz = 0;
        delta = oracle_joint_sweep(S1, S2, p, l1, l2, Om1, Om2, pairs, nc, &nnz);
        ++t;
        kkt = oracle_joint_kkt(S1, S2, Om1, Om2, p, l1, l2);
        if (history) {
            history[3 * (t - 1) + 0] = delta;
            history[3 * (t - 1) + 1] = kkt;
            history[3 * (t - 1) + 2] = oracle_joint_objective(S1, S2, Om1, Om2, p, l1, l2);
        }
        if (!first_delta && delta < delta_tol) first_delta = t;
        if (kkt <= tol) {
            status = 0;
            break;
        }
    }
    if (max_sweeps == 0 && kkt <= tol) status = 0;
    stats[0] = t;
    stats[1] = oracle_joint_objective(S1, S2, Om1, Om2, p, l1, l2);
    stats[2] = kkt;
    stats[3] = delta;
    stats[4] = first_delta;
    stats[5] = (double)nnz;
    free(pairs);
    return status;
}
