/*
 * Plain FP64 CPU oracle for greedy conditional selection and the KL-optimal
 * sparse inverse-Cholesky factor (Huan, Guinness, Katzfuss, Owhadi, Schaefer,
 * "Sparse inverse Cholesky factorization of dense kernel matrices by greedy
 * conditional selection").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; it exists so that the tests, the smoke check and the CPU
 * baseline of the benchmark have an independent, obviously-correct reference.
 * It shares no code, header or constant with the CUDA library.
 *
 * Every routine is a direct, unblocked transcription of the paper's
 * definitions, in the order the paper states them:
 *   - kernel entries (Section 2, Matern family, nugget on the diagonal);
 *   - reverse-maximin ordering (Section 2.2, eq. maximin), brute force O(N^2);
 *   - later-ordered nearest neighbours (Section 4 candidate sets), brute force;
 *   - supernode grouping (Section 6.1 grouping rule, lambda = 1.5);
 *   - single-target greedy selection by the Cholesky approach (Section 3.1,
 *     eqs. cond_select and obj_gp; Appendix B.1 / C.1);
 *   - multiple-target greedy selection with two partial Cholesky factors
 *     (Section 5.2, eq. greedy_mult; Appendix C.2);
 *   - KL-optimal column fill by a dense Cholesky solve (eq. L_col).
 * Compile with -ffp-contract=off so that a*b+c is never fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t dim;
    int32_t nu_x2;       /* 1, 3, 5 -> smoothness 1/2, 3/2, 5/2 */
    double length_scale; /* ell */
    double variance;     /* sigma^2 */
    double nugget;       /* added to the diagonal only */
    const double* dense; /* if non-NULL, Theta_{ab} = dense[a * dense_ld + b] instead */
    int64_t dense_ld;
} or_kernel;

/* ---------------------------------------------------------------- kernel -- */

/* Matern covariance at distance r (sqrt(2 nu) r / ell parameterisation). */
double or_matern(const or_kernel* kp, double r) {
    double s2 = kp->variance;
    if (kp->nu_x2 == 1) {
        return s2 * exp(-r / kp->length_scale);
    } else if (kp->nu_x2 == 3) {
        double t = sqrt(3.0) * r / kp->length_scale;
        return s2 * (1.0 + t) * exp(-t);
    } else {
        double t = sqrt(5.0) * r / kp->length_scale;
        return s2 * (1.0 + t + t * t / 3.0) * exp(-t);
    }
}

static double dist2(const double* pts, int dim, int64_t a, int64_t b) {
    double s = 0.0;
    for (int c = 0; c < dim; ++c) {
        double d = pts[a * dim + c] - pts[b * dim + c];
        s += d * d;
    }
    return s;
}

/* Theta_{ab} for rows a, b of the point array (nugget when a == b). */
double or_theta(const or_kernel* kp, const double* pts, int64_t a, int64_t b) {
    if (kp->dense) return kp->dense[a * kp->dense_ld + b];
    double v = or_matern(kp, sqrt(dist2(pts, kp->dim, a, b)));
    if (a == b) v += kp->nugget;
    return v;
}

/* ------------------------------------------------- reverse-maximin order -- */

/* eq. maximin: the last index is point 0; then, for positions N-2 .. 0, take the
 * unplaced point whose distance to the placed set is largest (ties: lowest point
 * index).  order[pos] = point index; ell2[pos] = squared distance from that point
 * to the points placed after it (INFINITY for the last position). */
void or_maximin(const double* pts, int64_t n, int dim, int64_t* order, double* ell2) {
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    char* placed = (char*)calloc((size_t)n, 1);
    placed[0] = 1;
    order[n - 1] = 0;
    ell2[n - 1] = INFINITY;
    for (int64_t j = 0; j < n; ++j) d[j] = dist2(pts, dim, j, 0);
    for (int64_t pos = n - 2; pos >= 0; --pos) {
        int64_t best = -1;
        for (int64_t j = 0; j < n; ++j) {
            if (placed[j]) continue;
            if (best < 0 || d[j] > d[best]) best = j;
        }
        order[pos] = best;
        ell2[pos] = d[best];
        placed[best] = 1;
        for (int64_t j = 0; j < n; ++j) {
            if (placed[j]) continue;
            double e = dist2(pts, dim, j, best);
            if (e < d[j]) d[j] = e;
        }
    }
    free(d);
    free(placed);
}

/* ------------------------------------------------------ nearest neighbours -- */

typedef struct { double key; int64_t pos; } keyed;

static int cmp_keyed(const void* a, const void* b) {
    const keyed* x = (const keyed*)a;
    const keyed* y = (const keyed*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->pos < y->pos) ? -1 : (x->pos > y->pos);
}

/* Candidates of a set of targets: the C points at positions >= first whose
 * smallest squared distance to any target is least, sorted by (that distance,
 * position).  pts are in elimination order.  Returns the count (<= C). */
int32_t or_knn_later(const double* pts, int64_t n, int dim, const int64_t* targets, int32_t m,
                     int64_t first, int32_t C, int32_t* out) {
    if (first >= n || C <= 0) return 0;
    int64_t cnt = n - first;
    keyed* all = (keyed*)malloc(sizeof(keyed) * (size_t)cnt);
    for (int64_t j = first; j < n; ++j) {
        double best = INFINITY;
        for (int32_t a = 0; a < m; ++a) {
            double e = dist2(pts, dim, j, targets[a]);
            if (e < best) best = e;
        }
        all[j - first].key = best;
        all[j - first].pos = j;
    }
    qsort(all, (size_t)cnt, sizeof(keyed), cmp_keyed);
    int32_t take = (cnt < C) ? (int32_t)cnt : C;
    for (int32_t t = 0; t < take; ++t) out[t] = (int32_t)all[t].pos;
    free(all);
    return take;
}

/* ---------------------------------------------------------------- groups -- */

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x < y) ? -1 : (x > y);
}

/* Supernodes by the grouping rule of Section 6.1: take the first position i not yet
 * in a group and group it with the positions j of its sparsity set s_i that are not
 * yet grouped and satisfy ell_j <= lambda ell_i (compared as squared lengths,
 * ell2_j <= lambda2 * ell2_i).  s_i is i plus its K nearest later points, scanned in
 * distance order; a group holds at most mmax points.  A second pass merges every
 * group smaller than mmin into the group formed just before it when the union holds
 * at most mmax points.  Members are written group after group, each group ascending
 * (this is the renumbered elimination order).  Returns the number of groups;
 * grp_ptr has n_groups + 1 entries. */
int64_t or_group(const double* pts, const double* ell2, int64_t n, int dim, int32_t K,
                 double lambda2, int32_t mmin, int32_t mmax, int64_t* members, int64_t* grp_ptr) {
    char* done = (char*)calloc((size_t)n, 1);
    int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
    int64_t* g = (int64_t*)malloc(sizeof(int64_t) * (size_t)(mmax + 1));
    int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t ng = 0, w = 0;
    first[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (done[i]) continue;
        int32_t gm = 0;
        g[gm++] = i;
        done[i] = 1;
        int32_t cnt = or_knn_later(pts, n, dim, &i, 1, i + 1, K, nb);
        for (int32_t t = 0; t < cnt && gm < mmax; ++t) {
            int64_t j = nb[t];
            if (done[j]) continue;
            if (ell2[j] <= lambda2 * ell2[i]) {
                g[gm++] = j;
                done[j] = 1;
            }
        }
        for (int32_t t = 0; t < gm; ++t) members[w++] = g[t];
        first[++ng] = w;
    }
    /* merge pass: groups are contiguous runs of members[], so merging a group into the
     * previous one only moves a boundary */
    int64_t out = 0;
    grp_ptr[0] = 0;
    for (int64_t q = 0; q < ng; ++q) {
        int64_t sz = first[q + 1] - first[q];
        if (out > 0 && sz < mmin && (first[q + 1] - grp_ptr[out - 1]) <= mmax) {
            grp_ptr[out] = first[q + 1];
        } else {
            grp_ptr[++out] = first[q + 1];
        }
    }
    for (int64_t q = 0; q < out; ++q)
        qsort(members + grp_ptr[q], (size_t)(grp_ptr[q + 1] - grp_ptr[q]), sizeof(int64_t), cmp_i64);
    free(done);
    free(nb);
    free(g);
    free(first);
    return out;
}

/* ----------------------------------------------------- dense linear algebra -- */

/* In-place lower Cholesky of the n x n row-major matrix A; returns 0 on success. */
static int chol_lower(double* A, int n) {
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int p = 0; p < j; ++p) s -= A[j * n + p] * A[j * n + p];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int p = 0; p < j; ++p) t -= A[i * n + p] * A[j * n + p];
            A[i * n + j] = t / d;
        }
        for (int p = j + 1; p < n; ++p) A[j * n + p] = 0.0;
    }
    return 0;
}

/* ------------------------------------------------ single-target selection -- */

/* Greedy conditional selection for one target (Section 3.1, Cholesky approach).
 * Rows 0..C-1 of the partial factor F are the candidates and row C the target.
 * Per step: score_j = cov_j^2 / var_j (eq. obj_gp) over candidates that are neither
 * selected nor exhausted (var_j < floor); the pivot q is the first maximiser (or
 * forced[step] when forced is non-NULL and forced[step] >= 0, an index into the
 * candidate list); the new column is u = (Theta[:, q] - F[:, :t] F[q, :t]^T) / sqrt(var_q)
 * (left-looking, Appendix B.1); then var_j -= u_j^2, cov_j -= u_j u_target,
 * var_target -= u_target^2 (eq. cond_select).
 * Outputs: sel[t] = position of the t-th pick; best[t] = the largest score at step t;
 * chosen[t] = the score of the pick; vtar[t] = target conditional variance after
 * t picks (vtar has room for k+1 values).  Returns the number of picks. */
int32_t or_select_single(const or_kernel* kp, const double* pts, int64_t target, const int32_t* cand,
                         int32_t C, int32_t k, double floor_, const int32_t* forced, int32_t* sel,
                         double* best, double* chosen, double* vtar) {
    int32_t R = C + 1;
    double* F = (double*)calloc((size_t)R * (size_t)(k > 0 ? k : 1), sizeof(double));
    double* var = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    double* cov = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    char* taken = (char*)calloc((size_t)(C > 0 ? C : 1), 1);
    for (int32_t j = 0; j < C; ++j) {
        var[j] = or_theta(kp, pts, cand[j], cand[j]);
        cov[j] = or_theta(kp, pts, target, cand[j]);
    }
    double vt = or_theta(kp, pts, target, target);
    if (vtar) vtar[0] = vt;
    int32_t t = 0;
    for (; t < k; ++t) {
        int32_t arg = -1;
        double bs = -INFINITY;
        for (int32_t j = 0; j < C; ++j) {
            if (taken[j] || var[j] < floor_) continue;
            double s = cov[j] * cov[j] / var[j];
            if (arg < 0 || s > bs) { arg = j; bs = s; }
        }
        if (arg < 0 || !(bs > 0.0)) break;
        int32_t q = (forced && forced[t] >= 0) ? forced[t] : arg;
        if (best) best[t] = bs;
        if (chosen) chosen[t] = cov[q] * cov[q] / var[q];
        double d = sqrt(var[q]);
        for (int32_t r = 0; r < R; ++r) {
            int64_t pr = (r < C) ? cand[r] : target;
            double num = or_theta(kp, pts, pr, cand[q]);
            for (int32_t tau = 0; tau < t; ++tau) num -= F[(size_t)r * k + tau] * F[(size_t)q * k + tau];
            F[(size_t)r * k + t] = num / d;
        }
        double ut = F[(size_t)C * k + t];
        for (int32_t j = 0; j < C; ++j) {
            double uj = F[(size_t)j * k + t];
            var[j] -= uj * uj;
            cov[j] -= uj * ut;
        }
        vt -= ut * ut;
        taken[q] = 1;
        sel[t] = cand[q];
        if (vtar) vtar[t + 1] = vt;
    }
    free(F);
    free(var);
    free(cov);
    free(taken);
    return t;
}

/* ---------------------------------------------- multiple-target selection -- */

/* Greedy selection shared by the m consecutive targets g0 .. g0+m-1 (Section 5.2,
 * Cholesky approach with two partial factors, Appendix C.2).  F2 first receives the
 * m target columns by left-looking (so var2_j = Theta_{jj | P}); then each step
 * scores candidates by var1_j / var2_j (eq. greedy_mult: selecting j changes
 * logdet Theta_{PP|I} by log var2_j - log var1_j), picks the first maximiser among
 * candidates that are neither selected nor exhausted (var2_j < floor), appends the
 * pivot column to F1 (conditioned on I) and to F2 (conditioned on P and I) and
 * downdates var1 and var2.  best/chosen as in or_select_single (scores are ratios).
 * Returns the number of picks, or -1 if the target block is not positive definite. */
int32_t or_select_multi(const or_kernel* kp, const double* pts, int64_t g0, int32_t m, const int32_t* cand,
                        int32_t C, int32_t k, double floor_, const int32_t* forced, int32_t* sel,
                        double* best, double* chosen) {
    int32_t R = C + m;          /* rows: candidates then targets */
    int32_t W2 = m + k;         /* columns of F2 */
    int32_t kk = (k > 0) ? k : 1;
    double* F1 = (double*)calloc((size_t)(C > 0 ? C : 1) * (size_t)kk, sizeof(double));
    double* F2 = (double*)calloc((size_t)R * (size_t)W2, sizeof(double));
    double* var1 = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    double* var2 = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    char* taken = (char*)calloc((size_t)(C > 0 ? C : 1), 1);
    int32_t t = 0;
    /* target columns of F2 */
    for (int32_t a = 0; a < m; ++a) {
        int32_t pr = C + a;
        double dv = or_theta(kp, pts, g0 + a, g0 + a);
        for (int32_t b = 0; b < a; ++b) dv -= F2[(size_t)pr * W2 + b] * F2[(size_t)pr * W2 + b];
        if (!(dv > 0.0)) { t = -1; goto done; }
        double d = sqrt(dv);
        for (int32_t r = 0; r < R; ++r) {
            int64_t prow = (r < C) ? cand[r] : g0 + (r - C);
            double num = or_theta(kp, pts, prow, g0 + a);
            for (int32_t b = 0; b < a; ++b) num -= F2[(size_t)r * W2 + b] * F2[(size_t)pr * W2 + b];
            F2[(size_t)r * W2 + a] = num / d;
        }
    }
    for (int32_t j = 0; j < C; ++j) {
        var1[j] = or_theta(kp, pts, cand[j], cand[j]);
        double v2 = var1[j];
        for (int32_t a = 0; a < m; ++a) v2 -= F2[(size_t)j * W2 + a] * F2[(size_t)j * W2 + a];
        var2[j] = v2;
    }
    for (t = 0; t < k; ++t) {
        int32_t arg = -1;
        double bs = -INFINITY;
        for (int32_t j = 0; j < C; ++j) {
            if (taken[j] || var2[j] < floor_) continue;
            double s = var1[j] / var2[j];
            if (arg < 0 || s > bs) { arg = j; bs = s; }
        }
        if (arg < 0) break;
        int32_t q = (forced && forced[t] >= 0) ? forced[t] : arg;
        if (best) best[t] = bs;
        if (chosen) chosen[t] = var1[q] / var2[q];
        double d1 = sqrt(var1[q]);
        double d2 = sqrt(var2[q]);
        for (int32_t j = 0; j < C; ++j) {
            double th = or_theta(kp, pts, cand[j], cand[q]);
            double n1 = th;
            for (int32_t tau = 0; tau < t; ++tau) n1 -= F1[(size_t)j * kk + tau] * F1[(size_t)q * kk + tau];
            F1[(size_t)j * kk + t] = n1 / d1;
            double n2 = th;
            for (int32_t tau = 0; tau < m + t; ++tau) n2 -= F2[(size_t)j * W2 + tau] * F2[(size_t)q * W2 + tau];
            F2[(size_t)j * W2 + m + t] = n2 / d2;
        }
        for (int32_t j = 0; j < C; ++j) {
            double u1 = F1[(size_t)j * kk + t];
            double u2 = F2[(size_t)j * W2 + m + t];
            var1[j] -= u1 * u1;
            var2[j] -= u2 * u2;
        }
        taken[q] = 1;
        sel[t] = cand[q];
    }
done:
    free(F1);
    free(F2);
    free(var1);
    free(var2);
    free(taken);
    return t;
}

/* --------------------------------------------------------------- the fill -- */

/* eq. L_col for the sparsity set s = (s[0], s[1], ..., s[n-1]) with s[0] the column's
 * own index: x = Theta_{ss}^{-1} e_1 by a dense Cholesky solve, L_{s,i} = x / sqrt(x_1).
 * Writes the n values into L (same order as s) and returns log Theta_{ii | s \ i}
 * = -log x_1 (eq. inverse_cond).  Returns NAN if Theta_{ss} is not positive definite. */
double or_fill_set(const or_kernel* kp, const double* pts, const int64_t* s, int32_t n, double* L) {
    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = 0; b < n; ++b) A[a * n + b] = or_theta(kp, pts, s[a], s[b]);
    double out = NAN;
    if (chol_lower(A, n) == 0) {
        /* forward: G y = e_1 */
        for (int32_t a = 0; a < n; ++a) {
            double r = (a == 0) ? 1.0 : 0.0;
            for (int32_t b = 0; b < a; ++b) r -= A[a * n + b] * y[b];
            y[a] = r / A[a * n + a];
        }
        /* backward: G^T x = y (x overwrites y) */
        for (int32_t a = n - 1; a >= 0; --a) {
            double r = y[a];
            for (int32_t b = a + 1; b < n; ++b) r -= A[b * n + a] * y[b];
            y[a] = r / A[a * n + a];
        }
        double sc = sqrt(y[0]);
        for (int32_t a = 0; a < n; ++a) L[a] = y[a] / sc;
        out = -log(y[0]);
    }
    free(A);
    free(y);
    return out;
}

/* Per-column fill of a single-target factor column i with selected positions sel
 * (any order): s = (i, sel sorted ascending).  rows receives s, L the values. */
double or_fill_column(const or_kernel* kp, const double* pts, int64_t i, const int32_t* sel, int32_t cnt,
                      int64_t* rows, double* L) {
    rows[0] = i;
    for (int32_t t = 0; t < cnt; ++t) rows[1 + t] = sel[t];
    qsort(rows + 1, (size_t)cnt, sizeof(int64_t), cmp_i64);
    return or_fill_set(kp, pts, rows, cnt + 1, L);
}

/* Aggregated fill of member a of the group g0 .. g0+m-1 (Section 5.1): its set is
 * (g0+a, g0+a+1, ..., g0+m-1, shared selections sorted ascending). */
double or_fill_member(const or_kernel* kp, const double* pts, int64_t g0, int32_t m, int32_t a,
                      const int32_t* sel, int32_t cnt, int64_t* rows, double* L) {
    int32_t n = 0;
    for (int32_t b = a; b < m; ++b) rows[n++] = g0 + b;
    for (int32_t t = 0; t < cnt; ++t) rows[n + t] = sel[t];
    qsort(rows + n, (size_t)cnt, sizeof(int64_t), cmp_i64);
    return or_fill_set(kp, pts, rows, n + cnt, L);
}

/* Dense kernel matrix of a list of rows (row-major n x n), for tests. */
void or_theta_matrix(const or_kernel* kp, const double* pts, const int64_t* idx, int32_t n, double* out) {
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = 0; b < n; ++b) out[(size_t)a * n + b] = or_theta(kp, pts, idx[a], idx[b]);
}

/* y = op(L) x for a CSC factor (col_ptr, row_idx, val), nrhs columns of x stored
 * row-major (x[r * nrhs + c]).  op 0: L x; op 1: L^T x; op 2: L (L^T x). */
void or_apply_factor(int64_t n, const int64_t* col_ptr, const int32_t* row_idx, const double* val, int32_t op,
                     const double* x, double* y, int32_t nrhs) {
    double* z = (double*)calloc((size_t)n * (size_t)nrhs, sizeof(double));
    if (op == 0) {
        memset(y, 0, sizeof(double) * (size_t)n * (size_t)nrhs);
        for (int64_t c = 0; c < n; ++c)
            for (int64_t p = col_ptr[c]; p < col_ptr[c + 1]; ++p)
                for (int32_t r = 0; r < nrhs; ++r) y[(int64_t)row_idx[p] * nrhs + r] += val[p] * x[c * nrhs + r];
    } else {
        for (int64_t c = 0; c < n; ++c)
            for (int64_t p = col_ptr[c]; p < col_ptr[c + 1]; ++p)
                for (int32_t r = 0; r < nrhs; ++r) z[c * nrhs + r] += val[p] * x[(int64_t)row_idx[p] * nrhs + r];
        if (op == 1) {
            memcpy(y, z, sizeof(double) * (size_t)n * (size_t)nrhs);
        } else {
            memset(y, 0, sizeof(double) * (size_t)n * (size_t)nrhs);
            for (int64_t c = 0; c < n; ++c)
                for (int64_t p = col_ptr[c]; p < col_ptr[c + 1]; ++p)
                    for (int32_t r = 0; r < nrhs; ++r) y[(int64_t)row_idx[p] * nrhs + r] += val[p] * z[c * nrhs + r];
        }
    }
    free(z);
}
