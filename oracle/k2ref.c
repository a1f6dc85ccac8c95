/*
 * Oracle for the enhanced Kogbetliantz SVD of order two (arXiv 2407.13116).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow CPU implementation written from the
 * paper, used by tests/, by the smoke check and by the CPU-baseline leg of the
 * benchmark.  It shares no code with the CUDA path and is never called by it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared (+ -fopenmp).
 * No x87: the wide type of eq. (EXT) is _Float128 (binary128), whose arithmetic is
 * IEEE binary128 with one rounding per operation on both x86_64 and aarch64.
 */
#define _GNU_SOURCE
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if !defined(__FLT128_MANT_DIG__) || __FLT128_MANT_DIG__ != 113
#error "the oracle needs an IEEE binary128 _Float128"
#endif
#if FLT_EVAL_METHOD != 0
#error "the oracle needs FLT_EVAL_METHOD == 0 (no excess precision)"
#endif

/* Branch flags reported in bits 8.. of info (shifted there by the store). */
#define K2REF_F_EXT      0x01  /* eq. (EXT) used for one element of R           */
#define K2REF_F_FALLBACK 0x02  /* t'=15 with r12''=0 or r22''=0 (Sect. 3.2.2)   */
#define K2REF_F_SWAP     0x04  /* r11 < r22: transpose-swap of eq. (RT)         */
#define K2REF_F_T2F2     0x08  /* tan(2phi) by eq. (t2f'')                      */
#define K2REF_F_T2F3     0x10  /* tan(2phi) by eq. (t2f''')                     */
#define K2REF_F_T2INF    0x20  /* tan(2phi) infinite, tan(phi) = 1 (Alg. 1)     */
#define K2REF_F_TPINF    0x40  /* tan(psi) infinite, eq. (tp') (Alg. 2)         */
#define K2REF_F_PSIG     0x80  /* singular values swapped by eq. (prec)         */
#define K2REF_F_T2NCR    0x400 /* tan(2phi) by Alg. 1's branch for a hypot that is not correctly rounded */

/* ------------------------------------------------------------------------- */
/* Unsigned big integers, little-endian base-2^32 limbs: exact squares and    */
/* sums for the midpoint comparisons of the correctly rounded hypot.          */
/* ------------------------------------------------------------------------- */
#define BN_LIMBS 168
typedef struct { int n; uint32_t w[BN_LIMBS]; } bn_t;

static void bn_trim(bn_t *a) { while (a->n > 0 && a->w[a->n - 1] == 0) --a->n; }

static void bn_set_u64(bn_t *a, uint64_t v)
{
    a->n = 2; a->w[0] = (uint32_t)v; a->w[1] = (uint32_t)(v >> 32); bn_trim(a);
}

static void bn_shl(bn_t *a, int k)
{
    if (a->n == 0 || k == 0) return;
    int q = k / 32, r = k % 32;
    int n = a->n + q + 1;
    if (n > BN_LIMBS) abort();
    uint32_t out[BN_LIMBS];
    memset(out, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; ++i) {
        uint64_t v = (uint64_t)a->w[i] << r;
        out[i + q] |= (uint32_t)v;
        out[i + q + 1] |= (uint32_t)(v >> 32);
    }
    memcpy(a->w, out, sizeof(uint32_t) * (size_t)n);
    a->n = n; bn_trim(a);
}

static void bn_add(bn_t *r, const bn_t *a, const bn_t *b)
{
    int n = a->n > b->n ? a->n : b->n;
    if (n + 1 > BN_LIMBS) abort();
    uint64_t c = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t v = c;
        if (i < a->n) v += a->w[i];
        if (i < b->n) v += b->w[i];
        r->w[i] = (uint32_t)v; c = v >> 32;
    }
    r->w[n] = (uint32_t)c; r->n = n + 1; bn_trim(r);
}

static void bn_mul(bn_t *r, const bn_t *a, const bn_t *b)
{
    int n = a->n + b->n;
    if (n > BN_LIMBS) abort();
    uint32_t out[BN_LIMBS];
    memset(out, 0, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < a->n; ++i) {
        uint64_t c = 0;
        for (int j = 0; j < b->n; ++j) {
            uint64_t v = (uint64_t)a->w[i] * b->w[j] + out[i + j] + c;
            out[i + j] = (uint32_t)v; c = v >> 32;
        }
        out[i + b->n] = (uint32_t)c;
    }
    memcpy(r->w, out, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    r->n = n; bn_trim(r);
}

static int bn_cmp(const bn_t *a, const bn_t *b)
{
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; --i)
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    return 0;
}

/* Operation counters (per thread) for the algorithmic operation count of the method:
 * additions/subtractions, multiplications, fmas, divisions, correctly rounded hypots,
 * evaluations of eq. (EXT) and square roots (those of the hypot that is not correctly
 * rounded).  Exact power-of-two scalings, comparisons and sign changes are not counted. */
enum { OP_ADD, OP_MUL, OP_FMA, OP_DIV, OP_HYP, OP_EXT, OP_SQRT, OP_N };
static _Thread_local long long k2ref_ops_d[OP_N], k2ref_ops_s[OP_N];
#define K2OP(k) ((void)(SFX(k2ref_ops)[k]++))

/* ------------------------------------------------------------------------- */
/* Double precision: p = 53, T = binary128.                                  */
/* ------------------------------------------------------------------------- */
#define R double
#define W _Float128
#define SFX(x) x##_d
#define P 53
#define E_MU (-1022)
#define E_NU 1023
#define EPSV 0x1p-53
#define NUV DBL_MAX
#define MUV DBL_MIN
#define FABS fabs
#define FMA fma
#define ILOGB ilogb
#define SCALBN scalbn
#define NEXTAFTER nextafter
#define FREXP frexp
#define LDEXP ldexp
#define WSQRT sqrtf128
#define RSQRT sqrt
#define RBITS uint64_t
#include "k2ref_body.inc"
#undef R
#undef W
#undef SFX
#undef P
#undef E_MU
#undef E_NU
#undef EPSV
#undef NUV
#undef MUV
#undef FABS
#undef FMA
#undef ILOGB
#undef SCALBN
#undef NEXTAFTER
#undef FREXP
#undef LDEXP
#undef WSQRT
#undef RSQRT
#undef RBITS

/* ------------------------------------------------------------------------- */
/* Single precision: p = 24, T = double.                                     */
/* ------------------------------------------------------------------------- */
#define R float
#define W double
#define SFX(x) x##_s
#define P 24
#define E_MU (-126)
#define E_NU 127
#define EPSV 0x1p-24f
#define NUV FLT_MAX
#define MUV FLT_MIN
#define FABS fabsf
#define FMA fmaf
#define ILOGB ilogbf
#define SCALBN scalbnf
#define NEXTAFTER nextafterf
#define FREXP frexpf
#define LDEXP ldexpf
#define WSQRT sqrt
#define RSQRT sqrtf
#define RBITS uint32_t
#include "k2ref_body.inc"

/* Read (and optionally reset) the calling thread's operation counters. */
void k2ref_opcount(int prec_double, long long out[7], int reset)
{
    long long *c = prec_double ? k2ref_ops_d : k2ref_ops_s;
    for (int k = 0; k < OP_N; ++k) { out[k] = c[k]; if (reset) c[k] = 0; }
}

/* ------------------------------------------------------------------------- */
/* Brute-force reference (not the method): closed-form singular values of     */
/* G = [[a,b],[c,d]] in binary128,                                            */
/*   sigma1 = (hypot(a+d, c-b) + hypot(a-d, b+c)) / 2,  sigma2 = |ad - bc| / sigma1, */
/* accurate to a few binary128 ulps over the whole double range (squares of    */
/* doubles stay normal in binary128).  Used only to pin the oracle.           */
/* ------------------------------------------------------------------------- */
typedef _Float128 q_t;

static q_t q_hypot(q_t x, q_t y) { return sqrtf128(x * x + y * y); }

static void q_sigma(q_t a, q_t b, q_t c, q_t d, q_t *s1, q_t *s2)
{
    q_t p = q_hypot(a + d, c - b), q = q_hypot(a - d, b + c);
    *s1 = (p + q) / 2;
    q_t det = a * d - b * c;
    if (det < 0) det = -det;
    *s2 = (*s1 == 0) ? 0 : det / *s1;
}

/* split a positive binary128 value as (hi + lo) * 2^e with 1 <= hi < 2 */
static void q_split(q_t x, int32_t *e, double *hi, double *lo)
{
    if (x == 0) { *e = 0; *hi = 0; *lo = 0; return; }
    int ex = ilogbf128(x);
    q_t m = scalbnf128(x, -ex);
    *e = ex; *hi = (double)m; *lo = (double)(m - (q_t)*hi);
}

/* G in column-major order (g11, g21, g12, g22); out: (e, hi, lo) for sigma1 then sigma2 */
void k2ref_brute_sigma(const double g[4], int32_t e[2], double hi[2], double lo[2])
{
    q_t s1, s2;
    q_sigma((q_t)g[0], (q_t)g[2], (q_t)g[1], (q_t)g[3], &s1, &s2);
    q_split(s1, &e[0], &hi[0], &lo[0]);
    q_split(s2, &e[1], &hi[1], &lo[1]);
}

/* Accuracy measures of Sect. 4, evaluated in binary128 for a batch of double results:
 * out[k*n+i], k = 0..4: re sigma1, re sigma2 (eq. relerr, 0/0 = 0), re U, re V (eq. ortho),
 * re G (eq. svdres).  Singular values are taken from their (e,f) form (Se, Sf). */
void k2ref_dmetrics(int64_t n, const double *G, int64_t ldg, const double *U, int64_t ldu,
                    const double *V, int64_t ldv, const int32_t *Se, const double *Sf, int64_t lds,
                    double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        q_t a = G[i], c = G[ldg + i], b = G[2 * ldg + i], d = G[3 * ldg + i];
        q_t t1, t2;
        q_sigma(a, b, c, d, &t1, &t2);
        q_t c1 = scalbnf128((q_t)Sf[i], Se[i]), c2 = scalbnf128((q_t)Sf[lds + i], Se[lds + i]);
        q_t r1 = (t1 == 0 && c1 == 0) ? 0 : fabsf128(t1 - c1) / t1;
        q_t r2 = (t2 == 0 && c2 == 0) ? 0 : (t2 == 0 ? (q_t)INFINITY : fabsf128(t2 - c2) / t2);
        q_t u[2][2] = { { U[i], U[2 * ldu + i] }, { U[ldu + i], U[3 * ldu + i] } };
        q_t v[2][2] = { { V[i], V[2 * ldv + i] }, { V[ldv + i], V[3 * ldv + i] } };
        q_t ou = 0, ov = 0;
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                q_t su = u[0][p] * u[0][q] + u[1][p] * u[1][q] - (p == q);
                q_t sv = v[0][p] * v[0][q] + v[1][p] * v[1][q] - (p == q);
                ou += su * su; ov += sv * sv;
            }
        /* residual ||G - U S V^T||_F / ||G||_F, computed with G scaled to avoid range issues */
        q_t gm[2][2] = { { a, b }, { c, d } }, sg[2] = { c1, c2 };
        q_t num = 0, den = 0;
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                q_t x = gm[p][q];
                for (int k = 0; k < 2; ++k) x -= u[p][k] * sg[k] * v[q][k];
                num += x * x; den += gm[p][q] * gm[p][q];
            }
        out[i] = (double)r1;
        out[n + i] = (double)r2;
        out[2 * n + i] = (double)sqrtf128(ou);
        out[3 * n + i] = (double)sqrtf128(ov);
        out[4 * n + i] = den == 0 ? (num == 0 ? 0.0 : INFINITY) : (double)sqrtf128(num / den);
    }
}
