/*
 * orc.h -- CPU oracle for multiple-precision (MP) matrix multiplication and LU.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Number model (arXiv 1410.1599, Sec. 1 and Sec. 3: MPFR-style binary
 * floating point with a p-bit mantissa, every operation correctly rounded):
 *
 *     x = (-1)^sign * M * 2^(exp - 32*nw)     with 2^(32*nw-1) <= M < 2^(32*nw)
 *
 * i.e. the mantissa is a fraction in [1/2, 1) held as nw little-endian 32-bit
 * words, nw = 2*ceil(p/64); the (32*nw - p) low bits of M are zero.  Zero has
 * exp == ORC_EXP_ZERO and M == 0, and keeps a sign (+0 / -0).  Every operation
 * returns the exact result rounded once to p bits, ties to even.
 *
 * Every exact intermediate is an ordinary big integer (orc_num.c); the
 * rounding routine is the textbook definition.  Nothing is blocked, fused
 * or reordered beyond what the paper's formulas state.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>
#include <stddef.h>

#define ORC_EXP_ZERO INT64_MIN
#define ORC_EXP_MAX  ((int64_t)1 << 62)
#define ORC_EXP_MIN  (-((int64_t)1 << 62))
#define ORC_MAXW     272            /* 32-bit words: mantissas up to 8704 bits */
#define ORC_MAXP     (32 * ORC_MAXW)

typedef struct {
    int8_t   sign;                  /* 0 = +, 1 = - */
    int64_t  exp;                   /* ORC_EXP_ZERO for zero */
    uint32_t m[ORC_MAXW];           /* little-endian words, nw of them used */
} orc_num;

/* Dense row-major matrix of p-bit numbers, one mantissa of nw words each. */
typedef struct {
    int64_t   rows, cols;
    int       p, nw;
    uint32_t *w;                    /* (r*cols + c)*nw + k */
    int64_t  *e;
    int8_t   *s;
} orc_mat;

enum { ORC_SIMPLE = 0, ORC_BLOCK = 1, ORC_STRASSEN = 2, ORC_WINOGRAD = 3 };
enum { ORC_PEEL = 0, ORC_MIXED = 1 };

/* ---- scalar arithmetic (orc_num.c) ---- */
int    orc_nw(int p);
void   orc_set_zero(orc_num *r, int sign);
int    orc_is_zero(const orc_num *x);
void   orc_copy(orc_num *r, const orc_num *x);
void   orc_mul(orc_num *r, const orc_num *a, const orc_num *b, int p);
void   orc_add(orc_num *r, const orc_num *a, const orc_num *b, int p);
void   orc_sub(orc_num *r, const orc_num *a, const orc_num *b, int p);
int    orc_div(orc_num *r, const orc_num *a, const orc_num *b, int p);  /* -1 if b == 0 */
int    orc_cmpabs(const orc_num *a, const orc_num *b, int p);
void   orc_round_to(orc_num *r, const orc_num *x, int p_from, int p_to);
void   orc_widen(orc_num *r, const orc_num *x, int p_from, int p_to);
double orc_to_double(const orc_num *x, int p);
int    orc_from_rational(orc_num *r, int64_t num, int64_t den, int p);

/* counters: every orc_mul / orc_add / orc_sub call while counting is enabled */
extern uint64_t orc_cnt_mul, orc_cnt_addsub;
extern int      orc_counting;
extern int      orc_range_error;

/* ---- matrices (orc_mat.c) ---- */
int  orc_mat_alloc(orc_mat *A, int64_t rows, int64_t cols, int p);
void orc_mat_free(orc_mat *A);
void orc_get(const orc_mat *A, int64_t r, int64_t c, orc_num *x);
void orc_put(orc_mat *A, int64_t r, int64_t c, const orc_num *x);
int  orc_mat_import(orc_mat *A, int64_t rows, int64_t cols, int p,
                    const uint64_t *limb, const int64_t *exp, const int8_t *sign,
                    int64_t ld, int64_t plane);
void orc_mat_export(const orc_mat *A, uint64_t *limb, int64_t *exp, int8_t *sign,
                    int64_t ld, int64_t plane);

/* ---- GEMM (orc_gemm.c) ---- */
int  orc_gemm(int algo, int cutoff, int policy, int nb,
              const orc_mat *A, const orc_mat *B, orc_mat *C);
void orc_count_model(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy,
                     uint64_t *mul, uint64_t *addsub);
int64_t orc_sample_set(int side, int algo, int64_t m, int64_t l, int64_t n, int cutoff,
                       int policy, int64_t x0, int64_t *out, int64_t cap);
int  orc_gemm_sampled(int algo, int cutoff, int policy, const orc_mat *A, const orc_mat *B,
                      const int64_t *rows, int64_t nr, const int64_t *cols, int64_t nc,
                      orc_mat *Csub);

/* ---- correctly rounded exact dot product (orc_num.c) ---- */
int  orc_dot_exact_vec(const orc_num *a, const orc_num *b, int64_t l, int p_in, int p_out,
                       orc_num *r);

/* ---- LU (orc_lu.c) ---- */
int  orc_lu(orc_mat *A, int64_t *piv, int panel, int algo, int cutoff, int policy, int pivoting);
int  orc_lu_solve(const orc_mat *LU, const int64_t *piv, const orc_mat *b, orc_mat *x);

#endif
