/*
 * orc_gemm.c -- oracle MP matrix multiplication C := AB, A m x l, B l x n
 * (arXiv 1410.1599 Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 *  Simple   (Eq. 1): c_ij = (((+0 + a_i1 b_1j) + a_i2 b_2j) + ... ), k ascending,
 *           every product and every sum rounded to p bits.
 *  Block    (Eq. 2): C_IJ accumulates A_IK B_KJ for block index K ascending,
 *           directly into C, so every c_ij sees the same k-ascending sequence
 *           as Simple (identical cost, Sec. 2, and identical bits).
 *  Strassen (Sec. 2, P1..P7 and the block form of C, each sum evaluated left
 *           to right as printed).
 *  Winograd (Sec. 2, Eqs. for S1..S8, M1..M7, T1, T2 and the block form of C).
 *  Recursion (Sec. 2 end): recurse while all of m, l, n exceed the cutoff
 *           n_min; below it the leaf product is Simple/Block.  Odd dimensions
 *           (Sec. 2 end, "dynamic padding and peeling"):
 *             ORC_PEEL : every odd dimension x is peeled to x-1;
 *             ORC_MIXED: x = 1 (mod 4) is peeled, x = 3 (mod 4) is padded to
 *                        x+1 with zeros (this is the reading under which the
 *                        operation counts reproduce Table 1).
 *           Peel fix-ups after the even part C' = A'B':
 *             l peeled : c_ij = RN(c_ij + RN(a_{i,l-1} b_{l-1,j})) on C';
 *             m peeled : last row of C by Simple over the whole l;
 *             n peeled : last column of C by Simple over the whole l.
 */
#include "orc.h"
#include <assert.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

/* Z = X[r0:r0+rows, c0:c0+cols], +0 outside X (zero padding) */
static void sub_copy(orc_mat *Z, const orc_mat *X, int64_t r0, int64_t c0,
                     int64_t rows, int64_t cols)
{
    orc_mat_alloc(Z, rows, cols, X->p);
    orc_num x;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            if (r0 + i < X->rows && c0 + j < X->cols) {
                orc_get(X, r0 + i, c0 + j, &x);
                orc_put(Z, i, j, &x);
            }
        }
}

/* Z = X + Y (op = +1) or X - Y (op = -1), elementwise, new matrix */
static void mat_addsub(orc_mat *Z, const orc_mat *X, const orc_mat *Y, int op)
{
    assert(X->rows == Y->rows && X->cols == Y->cols);
    orc_mat_alloc(Z, X->rows, X->cols, X->p);
    int64_t ne = X->rows * X->cols;
#pragma omp parallel for schedule(static) if (ne > 4096 && !orc_counting)
    for (int64_t t = 0; t < ne; ++t) {
        orc_num x, y, z;
        orc_get(X, t / X->cols, t % X->cols, &x);
        orc_get(Y, t / X->cols, t % X->cols, &y);
        if (op > 0) orc_add(&z, &x, &y, X->p); else orc_sub(&z, &x, &y, X->p);
        orc_put(Z, t / X->cols, t % X->cols, &z);
    }
}

/* c = (((+0 + a_r0 b_0c) + a_r1 b_1c) + ...) over k = 0..l-1 (Eq. 1) */
static void dot_simple(const orc_mat *A, int64_t r, const orc_mat *B, int64_t c, orc_num *out)
{
    orc_num acc, a, b, t;
    orc_set_zero(&acc, 0);
    for (int64_t k = 0; k < A->cols; ++k) {
        orc_get(A, r, k, &a);
        orc_get(B, k, c, &b);
        orc_mul(&t, &a, &b, A->p);
        orc_add(&acc, &acc, &t, A->p);
    }
    orc_copy(out, &acc);
}

/* Simple, Eq. 1.  C is allocated by the caller, m x n. */
static void gemm_simple(const orc_mat *A, const orc_mat *B, orc_mat *C)
{
    int64_t m = A->rows, n = B->cols;
#pragma omp parallel for schedule(dynamic, 1) if (m * n > 64 && !orc_counting)
    for (int64_t t = 0; t < m * n; ++t) {
        orc_num c;
        dot_simple(A, t / n, B, t % n, &c);
        orc_put(C, t / n, t % n, &c);
    }
}

/* Block, Eq. 2, square blocks of nb; C accumulates in place. */
static void gemm_block(const orc_mat *A, const orc_mat *B, orc_mat *C, int nb)
{
    int64_t m = A->rows, l = A->cols, n = B->cols;
    int p = A->p;
    orc_num z;
    orc_set_zero(&z, 0);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) orc_put(C, i, j, &z);
    for (int64_t I = 0; I < m; I += nb)
        for (int64_t J = 0; J < n; J += nb)
            for (int64_t K = 0; K < l; K += nb) {
                int64_t ie = I + nb < m ? I + nb : m;
                int64_t je = J + nb < n ? J + nb : n;
                int64_t ke = K + nb < l ? K + nb : l;
                for (int64_t i = I; i < ie; ++i)
                    for (int64_t j = J; j < je; ++j) {
                        orc_num c, a, b, t;
                        orc_get(C, i, j, &c);
                        for (int64_t k = K; k < ke; ++k) {
                            orc_get(A, i, k, &a);
                            orc_get(B, k, j, &b);
                            orc_mul(&t, &a, &b, p);
                            orc_add(&c, &c, &t, p);
                        }
                        orc_put(C, i, j, &c);
                    }
            }
}

/* even size used for the recursive part of an odd dimension */
static int64_t even_dim(int64_t x, int policy)
{
    if (x % 2 == 0) return x;
    if (policy == ORC_MIXED && x % 4 == 3) return x + 1;   /* pad */
    return x - 1;                                           /* peel */
}

/* ------------------------------------------------- one recursion step */

typedef int (*mul_fn)(void *ctx, const orc_mat *X, const orc_mat *Y, orc_mat *Z);

/*
 * One level of Strassen's algorithm (Sec. 2).  Operands are the quadrants
 * A11..A22, B11..B22; mul computes a child product.  Outputs C11..C22 are
 * allocated here.
 */
static int strassen_step(const orc_mat Aq[4], const orc_mat Bq[4], orc_mat Cq[4],
                         mul_fn mul, void *ctx)
{
    const orc_mat *A11 = &Aq[0], *A12 = &Aq[1], *A21 = &Aq[2], *A22 = &Aq[3];
    const orc_mat *B11 = &Bq[0], *B12 = &Bq[1], *B21 = &Bq[2], *B22 = &Bq[3];
    orc_mat P[7], X, Y, T;
    int rc = 0;
    /* P1 = (A11 + A22)(B11 + B22) */
    mat_addsub(&X, A11, A22, +1); mat_addsub(&Y, B11, B22, +1);
    rc |= mul(ctx, &X, &Y, &P[0]); orc_mat_free(&X); orc_mat_free(&Y);
    /* P2 = (A21 + A22) B11 */
    mat_addsub(&X, A21, A22, +1);
    rc |= mul(ctx, &X, B11, &P[1]); orc_mat_free(&X);
    /* P3 = A11 (B12 - B22) */
    mat_addsub(&Y, B12, B22, -1);
    rc |= mul(ctx, A11, &Y, &P[2]); orc_mat_free(&Y);
    /* P4 = A22 (B21 - B11) */
    mat_addsub(&Y, B21, B11, -1);
    rc |= mul(ctx, A22, &Y, &P[3]); orc_mat_free(&Y);
    /* P5 = (A11 + A12) B22 */
    mat_addsub(&X, A11, A12, +1);
    rc |= mul(ctx, &X, B22, &P[4]); orc_mat_free(&X);
    /* P6 = (A21 - A11)(B11 + B12) */
    mat_addsub(&X, A21, A11, -1); mat_addsub(&Y, B11, B12, +1);
    rc |= mul(ctx, &X, &Y, &P[5]); orc_mat_free(&X); orc_mat_free(&Y);
    /* P7 = (A12 - A22)(B21 + B22) */
    mat_addsub(&X, A12, A22, -1); mat_addsub(&Y, B21, B22, +1);
    rc |= mul(ctx, &X, &Y, &P[6]); orc_mat_free(&X); orc_mat_free(&Y);
    /* C11 = P1 + P4 - P5 + P7 (left to right) */
    mat_addsub(&T, &P[0], &P[3], +1); mat_addsub(&X, &T, &P[4], -1); orc_mat_free(&T);
    mat_addsub(&Cq[0], &X, &P[6], +1); orc_mat_free(&X);
    /* C12 = P3 + P5 */
    mat_addsub(&Cq[1], &P[2], &P[4], +1);
    /* C21 = P2 + P4 */
    mat_addsub(&Cq[2], &P[1], &P[3], +1);
    /* C22 = P1 + P3 - P2 + P6 (left to right) */
    mat_addsub(&T, &P[0], &P[2], +1); mat_addsub(&X, &T, &P[1], -1); orc_mat_free(&T);
    mat_addsub(&Cq[3], &X, &P[5], +1); orc_mat_free(&X);
    for (int i = 0; i < 7; ++i) orc_mat_free(&P[i]);
    return rc;
}

/* One level of Winograd's variant (Sec. 2, S1..S8, M1..M7, T1, T2, C). */
static int winograd_step(const orc_mat Aq[4], const orc_mat Bq[4], orc_mat Cq[4],
                         mul_fn mul, void *ctx)
{
    const orc_mat *A11 = &Aq[0], *A12 = &Aq[1], *A21 = &Aq[2], *A22 = &Aq[3];
    const orc_mat *B11 = &Bq[0], *B12 = &Bq[1], *B21 = &Bq[2], *B22 = &Bq[3];
    orc_mat S[9], M[8], T1, T2, U;
    int rc = 0;
    mat_addsub(&S[1], A21, A22, +1);      /* S1 = A21 + A22 */
    mat_addsub(&S[2], &S[1], A11, -1);    /* S2 = S1 - A11  */
    mat_addsub(&S[3], A11, A21, -1);      /* S3 = A11 - A21 */
    mat_addsub(&S[4], A12, &S[2], -1);    /* S4 = A12 - S2  */
    mat_addsub(&S[5], B12, B11, -1);      /* S5 = B12 - B11 */
    mat_addsub(&S[6], B22, &S[5], -1);    /* S6 = B22 - S5  */
    mat_addsub(&S[7], B22, B12, -1);      /* S7 = B22 - B12 */
    mat_addsub(&S[8], &S[6], B21, -1);    /* S8 = S6 - B21  */
    rc |= mul(ctx, &S[2], &S[6], &M[1]);  /* M1 = S2 S6   */
    rc |= mul(ctx, A11, B11, &M[2]);      /* M2 = A11 B11 */
    rc |= mul(ctx, A12, B21, &M[3]);      /* M3 = A12 B21 */
    rc |= mul(ctx, &S[3], &S[7], &M[4]);  /* M4 = S3 S7   */
    rc |= mul(ctx, &S[1], &S[5], &M[5]);  /* M5 = S1 S5   */
    rc |= mul(ctx, &S[4], B22, &M[6]);    /* M6 = S4 B22  */
    rc |= mul(ctx, A22, &S[8], &M[7]);    /* M7 = A22 S8  */
    for (int i = 1; i <= 8; ++i) orc_mat_free(&S[i]);
    mat_addsub(&T1, &M[1], &M[2], +1);    /* T1 = M1 + M2 */
    mat_addsub(&T2, &T1, &M[4], +1);      /* T2 = T1 + M4 */
    mat_addsub(&Cq[0], &M[2], &M[3], +1); /* C11 = M2 + M3 */
    mat_addsub(&U, &T1, &M[5], +1);       /* C12 = T1 + M5 + M6 */
    mat_addsub(&Cq[1], &U, &M[6], +1);
    orc_mat_free(&U);
    mat_addsub(&Cq[2], &T2, &M[7], -1);   /* C21 = T2 - M7 */
    mat_addsub(&Cq[3], &T2, &M[5], +1);   /* C22 = T2 + M5 */
    orc_mat_free(&T1); orc_mat_free(&T2);
    for (int i = 1; i <= 7; ++i) orc_mat_free(&M[i]);
    return rc;
}

/* one recursion level of algo, shared by the full and the sampled recursion */
int orc_gemm_step(int algo, const orc_mat Aq[4], const orc_mat Bq[4], orc_mat Cq[4],
                  mul_fn mul, void *ctx)
{
    return algo == ORC_STRASSEN ? strassen_step(Aq, Bq, Cq, mul, ctx)
                                : winograd_step(Aq, Bq, Cq, mul, ctx);
}

void orc_dot_simple_rc(const orc_mat *A, int64_t r, const orc_mat *B, int64_t c, orc_num *out)
{
    dot_simple(A, r, B, c, out);
}

/* ----------------------------------------------- full recursion (Sec. 2) */

typedef struct { int algo, cutoff, policy; } rec_cfg;

static int rec_full(void *ctx, const orc_mat *A, const orc_mat *B, orc_mat *C);

static int rec_full(void *vcfg, const orc_mat *A, const orc_mat *B, orc_mat *C)
{
    const rec_cfg *cfg = (const rec_cfg *)vcfg;
    int64_t m = A->rows, l = A->cols, n = B->cols;
    int p = A->p, rc = 0;
    orc_mat_alloc(C, m, n, p);
    if (!(m > cfg->cutoff && l > cfg->cutoff && n > cfg->cutoff)) {
        gemm_simple(A, B, C);                      /* leaf: Simple == Block bits */
        return 0;
    }
    int64_t M = even_dim(m, cfg->policy), Lr = even_dim(l, cfg->policy);
    int64_t N = even_dim(n, cfg->policy);
    int64_t h = M / 2, k = Lr / 2, w = N / 2;
    orc_mat Aq[4], Bq[4], Cq[4];
    sub_copy(&Aq[0], A, 0, 0, h, k); sub_copy(&Aq[1], A, 0, k, h, k);
    sub_copy(&Aq[2], A, h, 0, h, k); sub_copy(&Aq[3], A, h, k, h, k);
    sub_copy(&Bq[0], B, 0, 0, k, w); sub_copy(&Bq[1], B, 0, w, k, w);
    sub_copy(&Bq[2], B, k, 0, k, w); sub_copy(&Bq[3], B, k, w, k, w);
    rc = orc_gemm_step(cfg->algo, Aq, Bq, Cq, rec_full, vcfg);
    int64_t mr = M < m ? M : m, nr = N < n ? N : n;   /* real part of C' */
    orc_num x, a, b, t;
    for (int64_t i = 0; i < mr; ++i)
        for (int64_t j = 0; j < nr; ++j) {
            orc_get(&Cq[(i >= h) * 2 + (j >= w)], i % h, j % w, &x);
            orc_put(C, i, j, &x);
        }
    for (int q = 0; q < 4; ++q) { orc_mat_free(&Aq[q]); orc_mat_free(&Bq[q]); orc_mat_free(&Cq[q]); }
    if (Lr < l) {                                  /* l peeled: rank-1 fix-up */
        for (int64_t i = 0; i < mr; ++i)
            for (int64_t j = 0; j < nr; ++j) {
                orc_get(C, i, j, &x);
                orc_get(A, i, l - 1, &a);
                orc_get(B, l - 1, j, &b);
                orc_mul(&t, &a, &b, p);
                orc_add(&x, &x, &t, p);
                orc_put(C, i, j, &x);
            }
    }
    if (M < m)                                     /* m peeled: last row */
        for (int64_t j = 0; j < n; ++j) { dot_simple(A, m - 1, B, j, &x); orc_put(C, m - 1, j, &x); }
    if (N < n)                                     /* n peeled: last column */
        for (int64_t i = 0; i < mr; ++i) { dot_simple(A, i, B, n - 1, &x); orc_put(C, i, n - 1, &x); }
    return rc;
}

/*
 * C := AB by algo.  C must be unallocated; it is allocated m x n here.
 * nb is the Block tile (Block only).  Returns 0, or -1 on a bad argument.
 */
int orc_gemm(int algo, int cutoff, int policy, int nb,
             const orc_mat *A, const orc_mat *B, orc_mat *C)
{
    if (A->cols != B->rows || A->p != B->p) return -1;
    if (algo == ORC_SIMPLE) {
        orc_mat_alloc(C, A->rows, B->cols, A->p);
        gemm_simple(A, B, C);
        return 0;
    }
    if (algo == ORC_BLOCK) {
        if (nb < 1) return -1;
        orc_mat_alloc(C, A->rows, B->cols, A->p);
        gemm_block(A, B, C, nb);
        return 0;
    }
    if (algo != ORC_STRASSEN && algo != ORC_WINOGRAD) return -1;
    if (cutoff < 1) return -1;
    rec_cfg cfg = { algo, cutoff, policy };
    return rec_full(&cfg, A, B, C);
}

/* ------------------------------------------ operation-count model (Sec. 2) */

/*
 * Counts of MP multiplications and additions/subtractions performed by
 * orc_gemm, from the same control flow without arithmetic.  A leaf counts
 * m*l*n of each (Simple adds every product to an accumulator that starts at
 * +0).  A recursion level counts 7 child products plus, per half-size
 * operand, 5 + 5 + 8 (Strassen) or 4 + 4 + 7 (Winograd) matrix add/subs
 * (Sec. 2, Mul/Addsub recurrences), plus the peel fix-ups.
 */
void orc_count_model(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy,
                     uint64_t *mul, uint64_t *addsub)
{
    if (algo == ORC_SIMPLE || algo == ORC_BLOCK ||
        !(m > cutoff && l > cutoff && n > cutoff)) {
        *mul = (uint64_t)(m * l * n);
        *addsub = (uint64_t)(m * l * n);
        return;
    }
    int64_t M = even_dim(m, policy), Lr = even_dim(l, policy), N = even_dim(n, policy);
    int64_t h = M / 2, k = Lr / 2, w = N / 2;
    uint64_t cm, ca;
    orc_count_model(algo, h, k, w, cutoff, policy, &cm, &ca);
    int ca_ = algo == ORC_STRASSEN ? 5 : 4, cb_ = ca_, cc_ = algo == ORC_STRASSEN ? 8 : 7;
    uint64_t mu = 7 * cm;
    uint64_t ad = 7 * ca + (uint64_t)(ca_ * h * k + cb_ * k * w + cc_ * h * w);
    int64_t mr = M < m ? M : m, nr = N < n ? N : n;
    if (Lr < l) { mu += (uint64_t)(mr * nr); ad += (uint64_t)(mr * nr); }
    if (M < m)  { mu += (uint64_t)(l * n);   ad += (uint64_t)(l * n); }
    if (N < n)  { mu += (uint64_t)(mr * l);  ad += (uint64_t)(mr * l); }
    *mul = mu;
    *addsub = ad;
}
