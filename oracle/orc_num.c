/*
 * orc_num.c -- oracle scalar arithmetic: exact big-integer intermediates and
 * one correct rounding (round to nearest, ties to even) per operation.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * The paper computes with MPFR (Sec. 1, Sec. 3: binary mantissa of p bits,
 * 128..8192 bits), whose add, sub, mul and div return the exact result
 * rounded once.  Each function below forms the exact result as an ordinary
 * unsigned big integer times a power of two and hands it to orc_round_int,
 * which is the textbook definition of rounding to p bits.
 */
#include "orc.h"
#include <assert.h>
#include <stdlib.h>
#include <string.h>

uint64_t orc_cnt_mul = 0, orc_cnt_addsub = 0;
int orc_counting = 0;
int orc_range_error = 0;

#define BIGW (2 * ORC_MAXW + 8)     /* words of an exact intermediate */

/* ------------------------------------------------------------------------
 * Little-endian unsigned big integers on 32-bit words.
 * ---------------------------------------------------------------------- */
static int64_t big_bitlen(const uint32_t *a, int n)
{
    for (int i = n - 1; i >= 0; --i)
        if (a[i]) {
            int b = 0;
            uint32_t v = a[i];
            while (v) { ++b; v >>= 1; }
            return 32 * (int64_t)i + b;
        }
    return 0;
}

static int big_bit(const uint32_t *a, int n, int64_t i)
{
    if (i < 0 || i >= 32 * (int64_t)n) return 0;
    return (int)((a[i / 32] >> (i % 32)) & 1u);
}

/* word i of a, zero outside 0..n-1 */
static uint32_t big_word(const uint32_t *a, int n, int64_t i)
{
    return (i >= 0 && i < n) ? a[i] : 0u;
}

/* 1 if any bit with index < i is set */
static int big_any_below(const uint32_t *a, int n, int64_t i)
{
    if (i <= 0) return 0;
    int64_t full = i / 32;
    for (int64_t k = 0; k < full && k < n; ++k)
        if (a[k]) return 1;
    int rb = (int)(i % 32);
    if (rb && full < n && (a[full] & ((1u << rb) - 1u))) return 1;
    return 0;
}

static int big_is_zero(const uint32_t *a, int n)
{
    for (int i = 0; i < n; ++i) if (a[i]) return 0;
    return 1;
}

/* r (rn words) = a (an words) shifted right by s >= 0 bits */
static void big_shr(uint32_t *r, int rn, const uint32_t *a, int an, int64_t s)
{
    int64_t ws = s / 32;
    int bs = (int)(s % 32);
    for (int i = 0; i < rn; ++i) {
        uint32_t lo = big_word(a, an, i + ws);
        uint32_t hi = big_word(a, an, i + ws + 1);
        r[i] = bs ? (lo >> bs) | (hi << (32 - bs)) : lo;
    }
}

/* r (rn words) = a (an words) shifted left by s >= 0 bits, truncated to rn words */
static void big_shl(uint32_t *r, int rn, const uint32_t *a, int an, int64_t s)
{
    int64_t ws = s / 32;
    int bs = (int)(s % 32);
    for (int i = 0; i < rn; ++i) {
        uint32_t hi = big_word(a, an, i - ws);
        uint32_t lo = big_word(a, an, i - ws - 1);
        r[i] = bs ? (hi << bs) | (lo >> (32 - bs)) : hi;
    }
}

static void big_add(uint32_t *r, const uint32_t *a, const uint32_t *b, int n)
{
    uint64_t c = 0;
    for (int i = 0; i < n; ++i) {
        c += (uint64_t)a[i] + b[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    assert(c == 0);
}

/* r = a - b, requires a >= b */
static void big_sub(uint32_t *r, const uint32_t *a, const uint32_t *b, int n)
{
    int64_t br = 0;
    for (int i = 0; i < n; ++i) {
        int64_t d = (int64_t)a[i] - b[i] - br;
        br = d < 0;
        r[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
    }
    assert(br == 0);
}

static int big_cmp(const uint32_t *a, const uint32_t *b, int n)
{
    for (int i = n - 1; i >= 0; --i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

/* r (an+bn words) = a * b, schoolbook */
static void big_mul(uint32_t *r, const uint32_t *a, int an, const uint32_t *b, int bn)
{
    memset(r, 0, sizeof(uint32_t) * (an + bn));
    for (int i = 0; i < an; ++i) {
        uint64_t c = 0;
        for (int j = 0; j < bn; ++j) {
            c += (uint64_t)a[i] * b[j] + r[i + j];
            r[i + j] = (uint32_t)c;
            c >>= 32;
        }
        r[i + bn] = (uint32_t)c;
    }
}

/* binary restoring division: q = floor(num / den), rem = num mod den.
 * q has nn words, rem has dn words, den != 0 */
static void big_divmod(uint32_t *q, uint32_t *rem, const uint32_t *num, int nn,
                       const uint32_t *den, int dn)
{
    uint32_t r[BIGW + 1], t[BIGW + 1], d[BIGW + 1];
    int rn = dn + 1;
    memset(r, 0, sizeof(uint32_t) * rn);
    memset(d, 0, sizeof(uint32_t) * rn);
    memcpy(d, den, sizeof(uint32_t) * dn);
    memset(q, 0, sizeof(uint32_t) * nn);
    for (int64_t i = 32 * (int64_t)nn - 1; i >= 0; --i) {
        big_shl(t, rn, r, rn, 1);                 /* r = 2r + bit */
        t[0] |= (uint32_t)big_bit(num, nn, i);
        memcpy(r, t, sizeof(uint32_t) * rn);
        if (big_cmp(r, d, rn) >= 0) {
            big_sub(r, r, d, rn);
            q[i / 32] |= 1u << (i % 32);
        }
    }
    memcpy(rem, r, sizeof(uint32_t) * dn);
}

/* ------------------------------------------------------------------------
 * Number helpers
 * ---------------------------------------------------------------------- */
int orc_nw(int p) { return 2 * ((p + 63) / 64); }

void orc_set_zero(orc_num *r, int sign)
{
    memset(r->m, 0, sizeof r->m);
    r->sign = (int8_t)(sign ? 1 : 0);
    r->exp = ORC_EXP_ZERO;
}

int orc_is_zero(const orc_num *x) { return x->exp == ORC_EXP_ZERO; }

void orc_copy(orc_num *r, const orc_num *x) { if (r != x) memcpy(r, x, sizeof *r); }

static void check_range(orc_num *r)
{
    if (r->exp != ORC_EXP_ZERO && (r->exp > ORC_EXP_MAX || r->exp < ORC_EXP_MIN))
        orc_range_error = 1;
}

/*
 * r = RN_p(sign * (N + sticky*eps) * 2^E), N an n-word nonzero integer,
 * 0 < eps < 1.  A set sticky stands for a nonzero remainder below N's last
 * bit; it requires bitlen(N) >= p + 2, so that no rounding boundary lies
 * strictly between N and N + 1.
 *
 * With bl = bitlen(N): if bl <= p the value is exact.  Otherwise keep the top
 * p bits q = N >> (bl - p); the first dropped bit is the round bit and the OR
 * of the rest is the sticky bit; round up iff round && (sticky || q odd).
 * The result is q / 2^p * 2^(E + bl), renormalised if q carried to 2^p.
 */
static void orc_round_int(orc_num *r, int p, const uint32_t *N, int n, int64_t E,
                          int sticky, int sign)
{
    int nw = orc_nw(p);
    int64_t bl = big_bitlen(N, n);
    assert(bl > 0);
    assert(!sticky || bl >= p + 2);
    uint32_t q[BIGW];
    orc_num out;
    memset(&out, 0, sizeof out);
    if (bl <= p) {
        big_shl(out.m, nw, N, n, 32 * (int64_t)nw - bl);
    } else {
        int64_t s = bl - p;
        int qn = nw + 1;
        big_shr(q, qn, N, n, s);
        int rb = big_bit(N, n, s - 1);
        int st = sticky || big_any_below(N, n, s - 1);
        if (rb && (st || (q[0] & 1u))) {
            uint32_t one[BIGW];
            memset(one, 0, sizeof(uint32_t) * qn);
            one[0] = 1;
            big_add(q, q, one, qn);
        }
        if (big_bitlen(q, qn) > p) {              /* q == 2^p */
            uint32_t t[BIGW];
            big_shr(t, qn, q, qn, 1);
            memcpy(q, t, sizeof(uint32_t) * qn);
            bl += 1;
        }
        big_shl(out.m, nw, q, qn, 32 * (int64_t)nw - p);
    }
    out.exp = E + bl;
    out.sign = (int8_t)sign;
    check_range(&out);
    memcpy(r, &out, sizeof out);
}

/* |a| vs |b|: -1, 0, 1; zero is the smallest magnitude */
int orc_cmpabs(const orc_num *a, const orc_num *b, int p)
{
    int za = orc_is_zero(a), zb = orc_is_zero(b);
    if (za || zb) return za && zb ? 0 : (za ? -1 : 1);
    if (a->exp != b->exp) return a->exp < b->exp ? -1 : 1;
    return big_cmp(a->m, b->m, orc_nw(p));
}

/* r = RN_p(a * b).  The exact product of the mantissas has 2*nw words. */
void orc_mul(orc_num *r, const orc_num *a, const orc_num *b, int p)
{
    int nw = orc_nw(p);
    int sign = a->sign ^ b->sign;
    if (orc_counting) {
#pragma omp atomic
        orc_cnt_mul++;
    }
    if (orc_is_zero(a) || orc_is_zero(b)) { orc_set_zero(r, sign); return; }
    uint32_t P[BIGW];
    big_mul(P, a->m, nw, b->m, nw);
    orc_round_int(r, p, P, 2 * nw, a->exp + b->exp - 64 * (int64_t)nw, 0, sign);
}

/*
 * r = RN_p(a + b).
 * Zeros follow IEEE 754 round-to-nearest: (-0)+(-0) = -0, an exact zero sum of
 * nonzero terms (or of +0 and -0) is +0, and x + 0 = x.
 *
 * Let x be the operand of larger magnitude and d = ex - ey >= 0.  If
 * d >= p + 2 then |y| < 2^(ex-p-2) is below half the spacing of p-bit numbers
 * next to x on either side (2^(ex-p-1) above x; 2^(ex-p-2) below it when x is
 * a power of two), so RN_p(x + y) = x with no tie.  Otherwise the exact sum
 * (Mx * 2^d +- My) * 2^(ey - 32 nw) has at most 32 nw + p + 3 bits and is
 * rounded once.
 */
void orc_add(orc_num *r, const orc_num *a, const orc_num *b, int p)
{
    int nw = orc_nw(p);
    if (orc_counting) {
#pragma omp atomic
        orc_cnt_addsub++;
    }
    if (orc_is_zero(a) && orc_is_zero(b)) { orc_set_zero(r, a->sign & b->sign); return; }
    if (orc_is_zero(a)) { orc_copy(r, b); return; }
    if (orc_is_zero(b)) { orc_copy(r, a); return; }
    const orc_num *x = a, *y = b;
    if (orc_cmpabs(a, b, p) < 0) { x = b; y = a; }
    int64_t d = x->exp - y->exp;
    if (d >= p + 2) { orc_copy(r, x); return; }
    int n = 2 * nw + 4;
    uint32_t X[BIGW], Y[BIGW], S[BIGW];
    big_shl(X, n, x->m, nw, d);
    memset(Y, 0, sizeof(uint32_t) * n);
    memcpy(Y, y->m, sizeof(uint32_t) * nw);
    if (x->sign == y->sign) {
        big_add(S, X, Y, n);
    } else {
        big_sub(S, X, Y, n);                      /* |x| >= |y| */
        if (big_is_zero(S, n)) { orc_set_zero(r, 0); return; }
    }
    orc_round_int(r, p, S, n, y->exp - 32 * (int64_t)nw, 0, x->sign);
}

void orc_sub(orc_num *r, const orc_num *a, const orc_num *b, int p)
{
    orc_num nb;
    orc_copy(&nb, b);
    nb.sign ^= 1;
    orc_add(r, a, &nb, p);
}

/*
 * r = RN_p(a / b).  Q = floor(Ma * 2^(p+2) / Mb) lies in (2^(p+1), 2^(p+3)),
 * so it has at least p + 2 bits and a nonzero remainder is a valid sticky bit.
 */
int orc_div(orc_num *r, const orc_num *a, const orc_num *b, int p)
{
    int nw = orc_nw(p);
    int sign = a->sign ^ b->sign;
    if (orc_is_zero(b)) return -1;
    if (orc_is_zero(a)) { orc_set_zero(r, sign); return 0; }
    int n = 2 * nw + 2;
    uint32_t num[BIGW], q[BIGW], rem[BIGW];
    big_shl(num, n, a->m, nw, p + 2);
    big_divmod(q, rem, num, n, b->m, nw);
    orc_round_int(r, p, q, n, a->exp - b->exp - (p + 2), !big_is_zero(rem, nw), sign);
    return 0;
}

/* r = RN_{p_to}(x) for an x held at precision p_from */
void orc_round_to(orc_num *r, const orc_num *x, int p_from, int p_to)
{
    if (orc_is_zero(x)) { orc_set_zero(r, x->sign); return; }
    int nwf = orc_nw(p_from);
    orc_round_int(r, p_to, x->m, nwf, x->exp - 32 * (int64_t)nwf, 0, x->sign);
}

/* exact widening p_from <= p_to */
void orc_widen(orc_num *r, const orc_num *x, int p_from, int p_to)
{
    assert(p_from <= p_to);
    orc_round_to(r, x, p_from, p_to);
}

/* x as the nearest double (report only; not used by any computation) */
double orc_to_double(const orc_num *x, int p)
{
    if (orc_is_zero(x)) return x->sign ? -0.0 : 0.0;
    int nw = orc_nw(p);
    double v = 0.0;
    for (int i = nw - 1; i >= 0 && i >= nw - 4; --i)
        v += (double)x->m[i] * __builtin_ldexp(1.0, 32 * (i - nw));
    double e = (double)x->exp;
    if (e > 2000) e = 2000;
    if (e < -2000) e = -2000;
    v = __builtin_ldexp(v, (int)e);
    return x->sign ? -v : v;
}

/* r = RN_p(num / den) for small integers (den > 0) */
int orc_from_rational(orc_num *r, int64_t num, int64_t den, int p)
{
    orc_num a, b;
    uint32_t N[4];
    int sa = num < 0;
    uint64_t ua = sa ? (uint64_t)(-(num + 1)) + 1 : (uint64_t)num;
    if (den <= 0) return -1;
    if (ua == 0) { orc_set_zero(r, 0); return 0; }
    N[0] = (uint32_t)ua; N[1] = (uint32_t)(ua >> 32);
    orc_round_int(&a, p, N, 2, 0, 0, sa);
    N[0] = (uint32_t)(uint64_t)den; N[1] = (uint32_t)((uint64_t)den >> 32);
    orc_round_int(&b, p, N, 2, 0, 0, 0);
    return orc_div(r, &a, &b, p);
}

/* ------------------------------------------------------------------------
 * Correctly rounded exact dot product: RN_{p_out}(+0 + sum_k a_k b_k) with
 * the sum formed exactly (no intermediate rounding) and rounded once.  An
 * exact zero sum is +0.  Returns -1 if the exponent spread of the products
 * would need an accumulator wider than 2^24 bits.
 * ---------------------------------------------------------------------- */

/* acc (an words) += x (xn words) * 2^(32*off) */
static void big_add_at(uint32_t *acc, int64_t an, const uint32_t *x, int xn, int64_t off)
{
    uint64_t c = 0;
    for (int64_t i = 0; off + i < an; ++i) {
        if (i >= xn && !c) break;
        c += (uint64_t)acc[off + i] + (i < xn ? x[i] : 0u);
        acc[off + i] = (uint32_t)c;
        c >>= 32;
    }
    assert(c == 0);
}

int orc_dot_exact_vec(const orc_num *a, const orc_num *b, int64_t l, int p_in, int p_out,
                      orc_num *r)
{
    int nw = orc_nw(p_in);
    int64_t Emin = 0, Etop = 0;
    int any = 0;
    for (int64_t k = 0; k < l; ++k) {
        if (orc_is_zero(&a[k]) || orc_is_zero(&b[k])) continue;
        int64_t E = a[k].exp + b[k].exp - 64 * (int64_t)nw;
        if (!any || E < Emin) Emin = E;
        if (!any || E + 64 * nw > Etop) Etop = E + 64 * (int64_t)nw;
        any = 1;
    }
    if (!any) { orc_set_zero(r, 0); return 0; }
    int64_t width = Etop - Emin + 64;
    if (width > ((int64_t)1 << 24)) return -1;
    int64_t an = width / 32 + 2;
    uint32_t *pos = (uint32_t *)calloc((size_t)an, 4), *neg = (uint32_t *)calloc((size_t)an, 4);
    uint32_t P[BIGW], S[BIGW];
    for (int64_t k = 0; k < l; ++k) {
        if (orc_is_zero(&a[k]) || orc_is_zero(&b[k])) continue;
        int64_t E = a[k].exp + b[k].exp - 64 * (int64_t)nw;
        int64_t sh = E - Emin;
        big_mul(P, a[k].m, nw, b[k].m, nw);
        big_shl(S, 2 * nw + 1, P, 2 * nw, sh % 32);
        big_add_at((a[k].sign ^ b[k].sign) ? neg : pos, an, S, 2 * nw + 1, sh / 32);
    }
    int c = 0;
    for (int64_t i = an - 1; i >= 0 && !c; --i)
        if (pos[i] != neg[i]) c = pos[i] < neg[i] ? -1 : 1;
    if (c == 0) {
        orc_set_zero(r, 0);
    } else {
        uint32_t *big = c > 0 ? pos : neg, *small = c > 0 ? neg : pos;
        int64_t br = 0;
        for (int64_t i = 0; i < an; ++i) {
            int64_t d = (int64_t)big[i] - small[i] - br;
            br = d < 0;
            big[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
        }
        orc_round_int(r, p_out, big, (int)an, Emin, 0, c < 0);
    }
    free(pos);
    free(neg);
    return 0;
}
