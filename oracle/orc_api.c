/*
 * orc_api.c -- flat-pointer entry points of the oracle, for ctypes.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).  Matrices cross this boundary in the
 * interchange format of orc_mat.c (limb planes, exponent, sign; ld, plane).
 */
#include "orc.h"
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAT_ARGS(X) const uint64_t *X##l, const int64_t *X##e, const int8_t *X##s, int64_t X##ld, int64_t X##pl
#define OUT_ARGS(X) uint64_t *X##l, int64_t *X##e, int8_t *X##s, int64_t X##ld, int64_t X##pl

void orc_api_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_api_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_api_range_error(void)
{
    int e = orc_range_error;
    orc_range_error = 0;
    return e;
}

/* r[i] = x[i] op y[i] for i < count; op 0 add, 1 sub, 2 mul, 3 div.
 * Returns -1 on a division by zero (that entry is left untouched). */
int orc_api_scalar(int op, int p, int64_t count, MAT_ARGS(X), MAT_ARGS(Y), OUT_ARGS(R))
{
    orc_mat x, y, r;
    if (orc_mat_import(&x, 1, count, p, Xl, Xe, Xs, Xld, Xpl) ||
        orc_mat_import(&y, 1, count, p, Yl, Ye, Ys, Yld, Ypl)) return -2;
    orc_mat_alloc(&r, 1, count, p);
    int bad = 0;
    for (int64_t i = 0; i < count; ++i) {
        orc_num a, b, c;
        orc_get(&x, 0, i, &a);
        orc_get(&y, 0, i, &b);
        orc_set_zero(&c, 0);
        if (op == 0) orc_add(&c, &a, &b, p);
        else if (op == 1) orc_sub(&c, &a, &b, p);
        else if (op == 2) orc_mul(&c, &a, &b, p);
        else if (orc_div(&c, &a, &b, p)) bad = 1;
        orc_put(&r, 0, i, &c);
    }
    orc_mat_export(&r, Rl, Re, Rs, Rld, Rpl);
    orc_mat_free(&x); orc_mat_free(&y); orc_mat_free(&r);
    return bad ? -1 : 0;
}

/* r = RN_{p_to}(x) elementwise (p_to >= p_from widens exactly) */
int orc_api_convert(int p_from, int p_to, int64_t count, MAT_ARGS(X), OUT_ARGS(R))
{
    orc_mat x, r;
    if (orc_mat_import(&x, 1, count, p_from, Xl, Xe, Xs, Xld, Xpl)) return -2;
    orc_mat_alloc(&r, 1, count, p_to);
    for (int64_t i = 0; i < count; ++i) {
        orc_num a, c;
        orc_get(&x, 0, i, &a);
        orc_round_to(&c, &a, p_from, p_to);
        orc_put(&r, 0, i, &c);
    }
    orc_mat_export(&r, Rl, Re, Rs, Rld, Rpl);
    orc_mat_free(&x); orc_mat_free(&r);
    return 0;
}

int orc_api_to_double(int p, int64_t count, MAT_ARGS(X), double *out)
{
    orc_mat x;
    if (orc_mat_import(&x, 1, count, p, Xl, Xe, Xs, Xld, Xpl)) return -2;
    for (int64_t i = 0; i < count; ++i) {
        orc_num a;
        orc_get(&x, 0, i, &a);
        out[i] = orc_to_double(&a, p);
    }
    orc_mat_free(&x);
    return 0;
}

int orc_api_gemm(int algo, int cutoff, int policy, int nb, int64_t m, int64_t l, int64_t n,
                 int p, MAT_ARGS(A), MAT_ARGS(B), OUT_ARGS(C))
{
    orc_mat A, B, C;
    if (orc_mat_import(&A, m, l, p, Al, Ae, As, Ald, Apl)) return -2;
    if (orc_mat_import(&B, l, n, p, Bl, Be, Bs, Bld, Bpl)) { orc_mat_free(&A); return -2; }
    int rc = orc_gemm(algo, cutoff, policy, nb, &A, &B, &C);
    if (!rc) { orc_mat_export(&C, Cl, Ce, Cs, Cld, Cpl); orc_mat_free(&C); }
    orc_mat_free(&A); orc_mat_free(&B);
    return rc;
}

/* run orc_gemm single-threaded with the operation counters on */
int orc_api_gemm_counted(int algo, int cutoff, int policy, int nb, int64_t m, int64_t l,
                         int64_t n, int p, MAT_ARGS(A), MAT_ARGS(B), OUT_ARGS(C),
                         uint64_t *mul, uint64_t *addsub)
{
    orc_cnt_mul = orc_cnt_addsub = 0;
    orc_counting = 1;
    int rc = orc_api_gemm(algo, cutoff, policy, nb, m, l, n, p, Al, Ae, As, Ald, Apl,
                          Bl, Be, Bs, Bld, Bpl, Cl, Ce, Cs, Cld, Cpl);
    orc_counting = 0;
    *mul = orc_cnt_mul;
    *addsub = orc_cnt_addsub;
    return rc;
}

void orc_api_count_model(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy,
                         uint64_t *mul, uint64_t *addsub)
{
    orc_count_model(algo, m, l, n, cutoff, policy, mul, addsub);
}

int64_t orc_api_sample_set(int side, int algo, int64_t m, int64_t l, int64_t n, int cutoff,
                           int policy, int64_t x0, int64_t *out, int64_t cap)
{
    return orc_sample_set(side, algo, m, l, n, cutoff, policy, x0, out, cap);
}

/* C (nr x nc, written at C[i*Cld + j]) = (A B) on the closed rows x cols */
int orc_api_gemm_sampled(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n,
                         int p, MAT_ARGS(A), MAT_ARGS(B), const int64_t *rows, int64_t nr,
                         const int64_t *cols, int64_t nc, OUT_ARGS(C))
{
    orc_mat A, B, C;
    if (orc_mat_import(&A, m, l, p, Al, Ae, As, Ald, Apl)) return -2;
    if (orc_mat_import(&B, l, n, p, Bl, Be, Bs, Bld, Bpl)) { orc_mat_free(&A); return -2; }
    int rc = orc_gemm_sampled(algo, cutoff, policy, &A, &B, rows, nr, cols, nc, &C);
    if (!rc) { orc_mat_export(&C, Cl, Ce, Cs, Cld, Cpl); orc_mat_free(&C); }
    orc_mat_free(&A); orc_mat_free(&B);
    return rc;
}

/* C[i][j] = RN_{p_out}(exact sum_k a_ik b_kj) for the listed (rows x cols) */
int orc_api_dot_exact(int64_t m, int64_t l, int64_t n, int p, int p_out, MAT_ARGS(A),
                      MAT_ARGS(B), const int64_t *rows, int64_t nr, const int64_t *cols,
                      int64_t nc, OUT_ARGS(C))
{
    orc_mat A, B, C;
    if (orc_mat_import(&A, m, l, p, Al, Ae, As, Ald, Apl)) return -2;
    if (orc_mat_import(&B, l, n, p, Bl, Be, Bs, Bld, Bpl)) { orc_mat_free(&A); return -2; }
    orc_mat_alloc(&C, nr, nc, p_out);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int64_t t = 0; t < nr * nc; ++t) {
        int64_t i = rows[t / nc], j = cols[t % nc];
        orc_num *a = (orc_num *)malloc(sizeof(orc_num) * (size_t)(l ? l : 1));
        orc_num *b = (orc_num *)malloc(sizeof(orc_num) * (size_t)(l ? l : 1));
        orc_num r;
        for (int64_t k = 0; k < l; ++k) { orc_get(&A, i, k, &a[k]); orc_get(&B, k, j, &b[k]); }
        if (orc_dot_exact_vec(a, b, l, p, p_out, &r)) bad = 1;
        else orc_put(&C, t / nc, t % nc, &r);
        free(a); free(b);
    }
    if (!bad) orc_mat_export(&C, Cl, Ce, Cs, Cld, Cpl);
    orc_mat_free(&A); orc_mat_free(&B); orc_mat_free(&C);
    return bad ? -1 : 0;
}

/* in-place LU of the n x n matrix A (interchange arrays overwritten);
 * pivoting 0 gives the paper's unpivoted LU */
int orc_api_lu(int64_t n, int p, int panel, int algo, int cutoff, int policy, int pivoting,
               OUT_ARGS(A), int64_t *piv)
{
    orc_mat A;
    if (orc_mat_import(&A, n, n, p, Al, Ae, As, Ald, Apl)) return -2;
    int rc = orc_lu(&A, piv, panel, algo, cutoff, policy, pivoting);
    orc_mat_export(&A, Al, Ae, As, Ald, Apl);
    orc_mat_free(&A);
    return rc;
}

int orc_api_lu_solve(int64_t n, int p, MAT_ARGS(A), const int64_t *piv, MAT_ARGS(B),
                     OUT_ARGS(X))
{
    orc_mat A, b, x;
    if (orc_mat_import(&A, n, n, p, Al, Ae, As, Ald, Apl)) return -2;
    if (orc_mat_import(&b, n, 1, p, Bl, Be, Bs, Bld, Bpl)) { orc_mat_free(&A); return -2; }
    int rc = orc_lu_solve(&A, piv, &b, &x);
    if (!rc) { orc_mat_export(&x, Xl, Xe, Xs, Xld, Xpl); orc_mat_free(&x); }
    orc_mat_free(&A); orc_mat_free(&b);
    return rc;
}
