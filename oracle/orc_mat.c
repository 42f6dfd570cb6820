/*
 * orc_mat.c -- oracle matrix storage and the interchange format.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Interchange format (what the seeded input generators write and what the
 * tests read back): for a rows x cols matrix at precision p with
 * L = ceil(p/64) limbs,
 *     limb[k*plane + r*ld + c]  64-bit limb k of the mantissa, k = 0 most
 *                               significant; the mantissa fraction is
 *                               sum_k limb_k * 2^(-64(k+1))
 *     exp[r*ld + c]             exponent (INT64_MIN for zero)
 *     sign[r*ld + c]            0 = +, 1 = -
 */
#include "orc.h"
#include <stdlib.h>
#include <string.h>

int orc_mat_alloc(orc_mat *A, int64_t rows, int64_t cols, int p)
{
    A->rows = rows; A->cols = cols; A->p = p; A->nw = orc_nw(p);
    size_t ne = (size_t)(rows > 0 ? rows : 0) * (size_t)(cols > 0 ? cols : 0);
    size_t nz = ne ? ne : 1;
    A->w = (uint32_t *)calloc(nz * (size_t)A->nw, sizeof(uint32_t));
    A->e = (int64_t *)malloc(nz * sizeof(int64_t));
    A->s = (int8_t *)calloc(nz, 1);
    if (!A->w || !A->e || !A->s) { orc_mat_free(A); return -1; }
    for (size_t i = 0; i < ne; ++i) A->e[i] = ORC_EXP_ZERO;   /* +0 everywhere */
    return 0;
}

void orc_mat_free(orc_mat *A)
{
    free(A->w); free(A->e); free(A->s);
    A->w = NULL; A->e = NULL; A->s = NULL;
}

void orc_get(const orc_mat *A, int64_t r, int64_t c, orc_num *x)
{
    size_t i = (size_t)(r * A->cols + c);
    memset(x->m, 0, sizeof x->m);
    memcpy(x->m, A->w + i * A->nw, sizeof(uint32_t) * A->nw);
    x->exp = A->e[i];
    x->sign = A->s[i];
}

void orc_put(orc_mat *A, int64_t r, int64_t c, const orc_num *x)
{
    size_t i = (size_t)(r * A->cols + c);
    memcpy(A->w + i * A->nw, x->m, sizeof(uint32_t) * A->nw);
    A->e[i] = x->exp;
    A->s[i] = x->sign;
}

/* returns 0, or -1 if an entry is not a valid p-bit number */
int orc_mat_import(orc_mat *A, int64_t rows, int64_t cols, int p,
                   const uint64_t *limb, const int64_t *exp, const int8_t *sign,
                   int64_t ld, int64_t plane)
{
    if (orc_mat_alloc(A, rows, cols, p)) return -2;
    int L = A->nw / 2;
    int bad = 0;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            orc_num x;
            memset(&x, 0, sizeof x);
            int64_t off = r * ld + c;
            for (int k = 0; k < L; ++k) {
                uint64_t v = limb[k * plane + off];
                x.m[2 * (L - 1 - k)] = (uint32_t)v;
                x.m[2 * (L - 1 - k) + 1] = (uint32_t)(v >> 32);
            }
            x.exp = exp[off];
            x.sign = sign[off] ? 1 : 0;
            if (x.exp == ORC_EXP_ZERO) {
                for (int k = 0; k < A->nw; ++k) if (x.m[k]) bad = 1;
            } else {
                if (!(x.m[A->nw - 1] >> 31)) bad = 1;          /* normalised */
                for (int b = 0; b < 32 * A->nw - p; ++b)        /* below p: zero */
                    if ((x.m[b / 32] >> (b % 32)) & 1u) bad = 1;
            }
            orc_put(A, r, c, &x);
        }
    return bad ? -1 : 0;
}

void orc_mat_export(const orc_mat *A, uint64_t *limb, int64_t *exp, int8_t *sign,
                    int64_t ld, int64_t plane)
{
    int L = A->nw / 2;
    for (int64_t r = 0; r < A->rows; ++r)
        for (int64_t c = 0; c < A->cols; ++c) {
            orc_num x;
            orc_get(A, r, c, &x);
            int64_t off = r * ld + c;
            for (int k = 0; k < L; ++k)
                limb[k * plane + off] = (uint64_t)x.m[2 * (L - 1 - k)] |
                                        ((uint64_t)x.m[2 * (L - 1 - k) + 1] << 32);
            exp[off] = x.exp;
            sign[off] = x.sign;
        }
}
