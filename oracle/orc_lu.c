/*
 * orc_lu.c -- oracle blocked right-looking LU with partial pivoting and the
 * triangular solves (arXiv 1410.1599 Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * For each panel of K columns starting at j0 (Sec. 4, steps 1-3):
 *   1. panel factorisation, column k = j0 .. j0+K-1 in order:
 *        pivot row  = the first row i >= k with the largest |a_ik|
 *                     (row k itself when pivoting is off);
 *        swap rows k and pivot over all n columns;
 *        l_ik = RN(a_ik / a_kk) for i > k (one division, not a reciprocal);
 *        a_ij = RN(a_ij - RN(l_ik a_kj)) for i > k and panel columns j > k.
 *   2. U12 = L11^{-1} A12 (unit lower): for rows r of the panel and s < r
 *      ascending, a_rj = RN(a_rj - RN(l_rs a_sj)).
 *   3. A22 = RN(A22 - T), T = L21 U12 computed by the chosen GEMM algorithm
 *      (the underlined product of Sec. 4), one rounding for the subtraction.
 * The paper's LU has no pivoting (Sec. 4); partial pivoting is added here
 * and can be switched off, which gives the paper's procedure exactly.
 */
#include "orc.h"
#include <stdlib.h>
#include <string.h>

static void swap_rows(orc_mat *A, int64_t r1, int64_t r2)
{
    if (r1 == r2) return;
    orc_num x, y;
    for (int64_t c = 0; c < A->cols; ++c) {
        orc_get(A, r1, c, &x);
        orc_get(A, r2, c, &y);
        orc_put(A, r1, c, &y);
        orc_put(A, r2, c, &x);
    }
}

/* Returns 0, or k+1 if the pivot of column k is zero (A singular). */
int orc_lu(orc_mat *A, int64_t *piv, int panel, int algo, int cutoff, int policy, int pivoting)
{
    int64_t n = A->rows;
    int p = A->p;
    orc_num x, y, t, d;
    if (A->cols != n || panel < 1) return -1;
    for (int64_t j0 = 0; j0 < n; j0 += panel) {
        int64_t jb = (n - j0) < panel ? (n - j0) : panel;
        int64_t je = j0 + jb;
        /* 1. panel */
        for (int64_t k = j0; k < je; ++k) {
            int64_t pr = k;
            orc_num best;
            orc_get(A, k, k, &best);
            for (int64_t i = k + 1; pivoting && i < n; ++i) {
                orc_get(A, i, k, &x);
                if (orc_cmpabs(&x, &best, p) > 0) { pr = i; orc_copy(&best, &x); }
            }
            piv[k] = pr;
            if (orc_is_zero(&best)) return (int)(k + 1);
            swap_rows(A, k, pr);
            orc_get(A, k, k, &d);
#pragma omp parallel for schedule(static) private(x, y, t) if (n - k > 64)
            for (int64_t i = k + 1; i < n; ++i) {
                orc_num l, u;
                orc_get(A, i, k, &x);
                orc_div(&l, &x, &d, p);
                orc_put(A, i, k, &l);
                for (int64_t j = k + 1; j < je; ++j) {
                    orc_get(A, k, j, &u);
                    orc_get(A, i, j, &y);
                    orc_mul(&t, &l, &u, p);
                    orc_sub(&y, &y, &t, p);
                    orc_put(A, i, j, &y);
                }
            }
        }
        if (je >= n) break;
        /* 2. U12 rows j0..je-1, columns je..n-1 */
#pragma omp parallel for schedule(static) private(x, y, t) if (n - je > 64)
        for (int64_t j = je; j < n; ++j)
            for (int64_t r = j0 + 1; r < je; ++r) {
                orc_get(A, r, j, &y);
                for (int64_t s = j0; s < r; ++s) {
                    orc_num l;
                    orc_get(A, r, s, &l);
                    orc_get(A, s, j, &x);
                    orc_mul(&t, &l, &x, p);
                    orc_sub(&y, &y, &t, p);
                }
                orc_put(A, r, j, &y);
            }
        /* 3. A22 -= L21 U12 */
        orc_mat L21, U12, T;
        int64_t nr = n - je;
        orc_mat_alloc(&L21, nr, jb, p);
        orc_mat_alloc(&U12, jb, nr, p);
        for (int64_t i = 0; i < nr; ++i)
            for (int64_t c = 0; c < jb; ++c) { orc_get(A, je + i, j0 + c, &x); orc_put(&L21, i, c, &x); }
        for (int64_t r = 0; r < jb; ++r)
            for (int64_t c = 0; c < nr; ++c) { orc_get(A, j0 + r, je + c, &x); orc_put(&U12, r, c, &x); }
        int rc = orc_gemm(algo, cutoff, policy, 32, &L21, &U12, &T);
        orc_mat_free(&L21);
        orc_mat_free(&U12);
        if (rc) return -1;
#pragma omp parallel for schedule(static) private(x, y, t) if (nr > 64)
        for (int64_t i = 0; i < nr; ++i)
            for (int64_t c = 0; c < nr; ++c) {
                orc_get(A, je + i, je + c, &y);
                orc_get(&T, i, c, &t);
                orc_sub(&y, &y, &t, p);
                orc_put(A, je + i, je + c, &y);
            }
        orc_mat_free(&T);
    }
    return 0;
}

/*
 * Solve LU x = P b with the factors of orc_lu (the paper does not fix the
 * order of the substitutions; both are taken column by column):
 *   y = P b (the row exchanges of the factorisation, in order);
 *   forward, j = 0 .. n-1:      y_i = RN(y_i - RN(l_ij y_j)) for all i > j
 *                               (each y_i sees its terms in ascending j);
 *   backward, j = n-1 .. 0:     x_j = RN(y_j / u_jj), then
 *                               y_i = RN(y_i - RN(u_ij x_j)) for all i < j
 *                               (each y_i sees its terms in descending j).
 * b and x are n x 1.  Returns 0, or -1 on a zero diagonal.
 */
int orc_lu_solve(const orc_mat *LU, const int64_t *piv, const orc_mat *b, orc_mat *x)
{
    int64_t n = LU->rows;
    int p = LU->p;
    orc_num *v = (orc_num *)malloc(sizeof(orc_num) * (size_t)(n ? n : 1));
    orc_num a, t, u;
    for (int64_t i = 0; i < n; ++i) orc_get(b, i, 0, &v[i]);
    for (int64_t k = 0; k < n; ++k)
        if (piv[k] != k) { orc_num s = v[k]; v[k] = v[piv[k]]; v[piv[k]] = s; }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i) {
            orc_get(LU, i, j, &a);
            orc_mul(&t, &a, &v[j], p);
            orc_sub(&v[i], &v[i], &t, p);
        }
    for (int64_t j = n - 1; j >= 0; --j) {
        orc_get(LU, j, j, &u);
        if (orc_div(&t, &v[j], &u, p)) { free(v); return -1; }
        v[j] = t;
        for (int64_t i = 0; i < j; ++i) {
            orc_get(LU, i, j, &a);
            orc_mul(&t, &a, &v[j], p);
            orc_sub(&v[i], &v[i], &t, p);
        }
    }
    orc_mat_alloc(x, n, 1, p);
    for (int64_t i = 0; i < n; ++i) orc_put(x, i, 0, &v[i]);
    free(v);
    return 0;
}
