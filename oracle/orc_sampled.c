/*
 * orc_sampled.c -- the Strassen / Winograd recursion of orc_gemm.c evaluated
 * only on a closed subset of output rows and columns.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Why this is the same computation: in one recursion level (Sec. 2) the row
 * r' < h of every child operand on the A side is formed from rows r' and
 * r' + h of the parent's A only (h = half of the even row count), and each
 * output row r of the parent reads child row r mod h.  Hence if a row set R
 * of the parent contains, for every r in R that falls in the recursive part,
 * both r mod h and r mod h + h (when that is a real row), and R restricted to
 * [0, h) has the same property for the children ("closed"), then every value
 * the recursion computes on rows R depends only on rows R of the operands.
 * The same holds for columns of B.  Evaluating the same step functions as the
 * full recursion (orc_gemm_step in orc_gemm.c) on those rows and columns
 * yields bit-identical values for the sampled outputs, at a cost of about
 * 2^depth rows instead of m.
 */
#include "orc.h"
#include <assert.h>
#include <stdlib.h>
#include <string.h>

int orc_gemm_step(int algo, const orc_mat Aq[4], const orc_mat Bq[4], orc_mat Cq[4],
                  int (*mul)(void *, const orc_mat *, const orc_mat *, orc_mat *),
                  void *ctx);
void orc_dot_simple_rc(const orc_mat *A, int64_t r, const orc_mat *B, int64_t c, orc_num *out);

static int64_t even_dim(int64_t x, int policy)
{
    if (x % 2 == 0) return x;
    if (policy == ORC_MIXED && x % 4 == 3) return x + 1;
    return x - 1;
}

/* sorted set of int64 in a caller-sized buffer */
typedef struct { int64_t *v; int64_t n, cap; } iset;

static int iset_has(const iset *s, int64_t x)
{
    for (int64_t i = 0; i < s->n; ++i) if (s->v[i] == x) return 1;
    return 0;
}

static int iset_add(iset *s, int64_t x)
{
    if (iset_has(s, x)) return 0;
    if (s->n >= s->cap) return -1;
    int64_t i = s->n++;
    while (i > 0 && s->v[i - 1] > x) { s->v[i] = s->v[i - 1]; --i; }
    s->v[i] = x;
    return 0;
}

static int64_t iset_index(const iset *s, int64_t x)
{
    for (int64_t i = 0; i < s->n; ++i) if (s->v[i] == x) return i;
    return -1;
}

/*
 * Closure of S (in place).  side 0: rows of A (dimension m, halves h),
 * side 1: columns of B (dimension n, halves w).
 */
static int closure(int side, int64_t m, int64_t l, int64_t n, int cutoff, int policy, iset *S)
{
    if (!(m > cutoff && l > cutoff && n > cutoff)) return 0;
    int64_t x = side ? n : m;
    int64_t X = even_dim(x, policy);
    int64_t half = X / 2;
    int64_t xr = X < x ? X : x;                 /* real rows of the recursive part */
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)S->cap);
    iset C = { buf, 0, S->cap };
    for (int64_t i = 0; i < S->n; ++i)
        if (S->v[i] < xr && iset_add(&C, S->v[i] % half)) { free(buf); return -1; }
    int rc = closure(side, even_dim(m, policy) / 2, even_dim(l, policy) / 2,
                     even_dim(n, policy) / 2, cutoff, policy, &C);
    for (int64_t i = 0; !rc && i < C.n; ++i) {
        if (iset_add(S, C.v[i])) rc = -1;
        if (!rc && C.v[i] + half < x && iset_add(S, C.v[i] + half)) rc = -1;
    }
    free(buf);
    return rc;
}

/* number of closed rows (side 0) / columns (side 1) written to out, or -1 */
int64_t orc_sample_set(int side, int algo, int64_t m, int64_t l, int64_t n, int cutoff,
                       int policy, int64_t x0, int64_t *out, int64_t cap)
{
    iset S = { out, 0, cap };
    if (iset_add(&S, x0)) return -1;
    if (algo == ORC_STRASSEN || algo == ORC_WINOGRAD)
        if (closure(side, m, l, n, cutoff, policy, &S)) return -1;
    return S.n;
}

typedef struct {
    int algo, cutoff, policy;
    int64_t m, l, n;           /* dimensions of the node this context multiplies for */
    const iset *R, *Cc;        /* its closed row and column sets */
} sub_ctx;

static int rec_sub(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n,
                   const iset *R, const orc_mat *Asub, const iset *Cs, const orc_mat *Bsub,
                   orc_mat *Csub);

static int sub_mul(void *vctx, const orc_mat *X, const orc_mat *Y, orc_mat *Z)
{
    const sub_ctx *c = (const sub_ctx *)vctx;
    return rec_sub(c->algo, c->cutoff, c->policy, c->m, c->l, c->n, c->R, X, c->Cc, Y, Z);
}

/*
 * C restricted to rows R x columns Cs of the node product A (m x l) B (l x n),
 * given Asub = rows R of A (|R| x l) and Bsub = columns Cs of B (l x |Cs|).
 */
static int rec_sub(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n,
                   const iset *R, const orc_mat *Asub, const iset *Cs, const orc_mat *Bsub,
                   orc_mat *Csub)
{
    int p = Asub->p, rc = 0;
    orc_mat_alloc(Csub, R->n, Cs->n, p);
    orc_num x, a, b, t;
    if (!(m > cutoff && l > cutoff && n > cutoff)) {
        for (int64_t i = 0; i < R->n; ++i)
            for (int64_t j = 0; j < Cs->n; ++j) {
                orc_dot_simple_rc(Asub, i, Bsub, j, &x);
                orc_put(Csub, i, j, &x);
            }
        return 0;
    }
    int64_t M = even_dim(m, policy), Lr = even_dim(l, policy), N = even_dim(n, policy);
    int64_t h = M / 2, k = Lr / 2, w = N / 2;
    int64_t mr = M < m ? M : m, nr = N < n ? N : n;
    int64_t rbuf[4096], cbuf[4096];
    iset R2 = { rbuf, 0, 4096 }, C2 = { cbuf, 0, 4096 };
    for (int64_t i = 0; i < R->n; ++i) if (R->v[i] < h) iset_add(&R2, R->v[i]);
    for (int64_t j = 0; j < Cs->n; ++j) if (Cs->v[j] < w) iset_add(&C2, Cs->v[j]);
    orc_mat Aq[4], Bq[4], Cq[4];
    for (int q = 0; q < 4; ++q) {
        orc_mat_alloc(&Aq[q], R2.n, k, p);
        orc_mat_alloc(&Bq[q], k, C2.n, p);
    }
    /* A quadrants on rows R2: (q / 2) selects the row half, (q % 2) the column half */
    for (int q = 0; q < 4; ++q)
        for (int64_t i = 0; i < R2.n; ++i) {
            int64_t r = R2.v[i] + (q / 2) * h;
            if (r >= m) continue;                              /* zero padding */
            int64_t ri = iset_index(R, r);
            assert(ri >= 0);
            for (int64_t c = 0; c < k; ++c) {
                int64_t cc = c + (q % 2) * k;
                if (cc >= l) continue;
                orc_get(Asub, ri, cc, &x);
                orc_put(&Aq[q], i, c, &x);
            }
        }
    for (int q = 0; q < 4; ++q)
        for (int64_t j = 0; j < C2.n; ++j) {
            int64_t c = C2.v[j] + (q % 2) * w;
            if (c >= n) continue;
            int64_t cj = iset_index(Cs, c);
            assert(cj >= 0);
            for (int64_t r = 0; r < k; ++r) {
                int64_t rr = r + (q / 2) * k;
                if (rr >= l) continue;
                orc_get(Bsub, rr, cj, &x);
                orc_put(&Bq[q], r, j, &x);
            }
        }
    sub_ctx ctx = { algo, cutoff, policy, h, k, w, &R2, &C2 };
    rc = orc_gemm_step(algo, Aq, Bq, Cq, sub_mul, &ctx);
    for (int64_t i = 0; i < R->n; ++i)
        for (int64_t j = 0; j < Cs->n; ++j) {
            int64_t r = R->v[i], c = Cs->v[j];
            if (M < m && r == m - 1) {
                orc_dot_simple_rc(Asub, i, Bsub, j, &x);        /* peeled last row */
            } else if (N < n && c == n - 1) {
                orc_dot_simple_rc(Asub, i, Bsub, j, &x);        /* peeled last column */
            } else {
                assert(r < mr && c < nr);
                orc_get(&Cq[(r >= h) * 2 + (c >= w)], iset_index(&R2, r % h),
                        iset_index(&C2, c % w), &x);
                if (Lr < l) {                                   /* peeled l: rank-1 */
                    orc_get(Asub, i, l - 1, &a);
                    orc_get(Bsub, l - 1, j, &b);
                    orc_mul(&t, &a, &b, p);
                    orc_add(&x, &x, &t, p);
                }
            }
            orc_put(Csub, i, j, &x);
        }
    for (int q = 0; q < 4; ++q) { orc_mat_free(&Aq[q]); orc_mat_free(&Bq[q]); orc_mat_free(&Cq[q]); }
    return rc;
}

/*
 * Csub (|rows| x |cols|, allocated here) = (A B) on rows x cols for algo, where
 * rows / cols are closed sets from orc_sample_set.  Returns 0, -1 on bad input.
 */
int orc_gemm_sampled(int algo, int cutoff, int policy, const orc_mat *A, const orc_mat *B,
                     const int64_t *rows, int64_t nr, const int64_t *cols, int64_t nc,
                     orc_mat *Csub)
{
    int64_t m = A->rows, l = A->cols, n = B->cols;
    if (A->cols != B->rows || nr > 4096 || nc > 4096) return -1;
    int64_t rb[4096], cb[4096];
    iset R = { rb, 0, 4096 }, C = { cb, 0, 4096 };
    for (int64_t i = 0; i < nr; ++i) if (rows[i] < 0 || rows[i] >= m || iset_add(&R, rows[i])) return -1;
    for (int64_t j = 0; j < nc; ++j) if (cols[j] < 0 || cols[j] >= n || iset_add(&C, cols[j])) return -1;
    if (R.n != nr || C.n != nc) return -1;
    if (algo == ORC_STRASSEN || algo == ORC_WINOGRAD) {
        /* the given sets must already be closed */
        int64_t tb[4096];
        iset T = { tb, 0, 4096 };
        for (int64_t i = 0; i < R.n; ++i) iset_add(&T, R.v[i]);
        if (closure(0, m, l, n, cutoff, policy, &T) || T.n != R.n) return -1;
        T.n = 0;
        for (int64_t j = 0; j < C.n; ++j) iset_add(&T, C.v[j]);
        if (closure(1, m, l, n, cutoff, policy, &T) || T.n != C.n) return -1;
    }
    orc_mat Asub, Bsub;
    orc_mat_alloc(&Asub, R.n, l, A->p);
    orc_mat_alloc(&Bsub, l, C.n, A->p);
    orc_num x;
    for (int64_t i = 0; i < R.n; ++i)
        for (int64_t k = 0; k < l; ++k) { orc_get(A, R.v[i], k, &x); orc_put(&Asub, i, k, &x); }
    for (int64_t k = 0; k < l; ++k)
        for (int64_t j = 0; j < C.n; ++j) { orc_get(B, k, C.v[j], &x); orc_put(&Bsub, k, j, &x); }
    int rc;
    if (algo == ORC_STRASSEN || algo == ORC_WINOGRAD) {
        rc = rec_sub(algo, cutoff, policy, m, l, n, &R, &Asub, &C, &Bsub, Csub);
    } else {
        orc_mat_alloc(Csub, R.n, C.n, A->p);
        for (int64_t i = 0; i < R.n; ++i)
            for (int64_t j = 0; j < C.n; ++j) {
                orc_dot_simple_rc(&Asub, i, &Bsub, j, &x);
                orc_put(Csub, i, j, &x);
            }
        rc = 0;
    }
    orc_mat_free(&Asub);
    orc_mat_free(&Bsub);
    return rc;
}
