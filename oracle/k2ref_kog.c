/*
 * Oracle of the batched n x n Kogbetliantz SVD, TEST INFRASTRUCTURE ONLY.
 *
 * Eq. (SVD) of Sect. 1: G_{k+1} = U_k^T G_k V_k, U_{k+1} = U_k U_k-hat, V_{k+1} = V_k V_k-hat,
 * where a step transforms the disjoint pivot pairs (i, j) of the parallel modulus
 * strategy: step k = 0, ..., n-1 of a sweep takes all pairs i < j with i + j = k (mod n).
 * Each pivot [[g_ii, g_ij], [g_ji, g_jj]] is decomposed by the 2x2 method of Sect. 3.
 * The paper leaves the rest open; the readings taken (also listed in the design notes):
 *  - all pivot SVDs of a step use G_k; then all row rotations are applied, then all
 *    column rotations, then U and V are updated, and the pivot blocks are set to
 *    diag(sigma1, sigma2) with exact zeros off the diagonal;
 *  - every rotated pair (x, y) becomes (fma(m21, y, m11 x), fma(m22, y, m12 x)) with m the
 *    2x2 factor in column-major order (m11, m21, m12, m22);
 *  - G is first scaled by the power of two that brings its largest element into [1/2, 1),
 *    so that no square in the norms can overflow (the singular values are scaled back);
 *  - off(G) = sqrt(sum over columns c of (sum over rows r != c, in increasing r, of
 *    fma-accumulated g_rc^2)), the column sums added in increasing c; the same order gives
 *    ||G||_F; the iteration stops when off(G) < tol_factor * n * eps * ||G||_F (eps = 2^-52
 *    or 2^-23) or after max_sweeps sweeps;
 *  - at exit a negative diagonal element g_ii (possible when the test holds before a
 *    sweep has touched it) is negated together with column i of U (signs go to the left,
 *    as in Sect. 3.1), then the diagonal is sorted into descending order (stable),
 *    permuting U and V.
 * The dynamic ordering (Sect. 1 names it as a candidate parallel strategy) replaces the
 * modulus pairs of a step: every pair i < j gets the weight w_ij = fma(g_ji, g_ji, g_ij^2)
 * from G_k, the pairs are ranked by decreasing weight (ties: smaller i, then smaller j),
 * and the ranked list is scanned once, each pair whose two indices are both still free
 * being taken, until floor(n/2) pairs are taken.  A "sweep" is still n such steps, with
 * the same convergence test before each.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void k2ref_pivot_d(double g11, double g21, double g12, double g22, double u[4], double v[4], double s[2]);
void k2ref_pivot_s(float g11, float g21, float g12, float g22, float u[4], float v[4], float s[2]);

#define KOG_BODY(R, SFX, PIVOT, FMA, SQRT, SCALBN, ILOGB, EPS)                                      \
typedef struct { R w; int i, j; } SFX(wpair);                                                     \
static int SFX(wcmp)(const void *pa, const void *pb)          /* decreasing w, then (i, j) */     \
{                                                                                                 \
    const SFX(wpair) *a = (const SFX(wpair) *)pa, *b = (const SFX(wpair) *)pb;                    \
    if (a->w != b->w) return a->w > b->w ? -1 : 1;                                                \
    if (a->i != b->i) return a->i < b->i ? -1 : 1;                                                \
    return a->j < b->j ? -1 : (a->j > b->j);                                                      \
}                                                                                                 \
/* The pairs of one step of the dynamic ordering from G (column-major, order n): np pairs */    \
/* (pi[p], pj[p]) in the order taken. */                                                        \
int SFX(k2ref_dyn_pairs)(int32_t n, const R *G, int32_t *pi, int32_t *pj)                         \
{                                                                                                 \
    size_t m = (size_t)n * (size_t)(n - 1) / 2, q = 0;                                            \
    SFX(wpair) *L = (SFX(wpair) *)malloc(sizeof(SFX(wpair)) * (m ? m : 1));                       \
    char *used = (char *)calloc((size_t)n, 1);                                                    \
    for (int i = 0; i < n; ++i)                                                                   \
        for (int j = i + 1; j < n; ++j) {                                                         \
            R gij = G[(size_t)j * n + i], gji = G[(size_t)i * n + j];                             \
            L[q].w = FMA(gji, gji, gij * gij); L[q].i = i; L[q].j = j; ++q;                       \
        }                                                                                         \
    qsort(L, m, sizeof(SFX(wpair)), SFX(wcmp));                                                   \
    int np = 0;                                                                                   \
    for (size_t e = 0; e < m && np < n / 2; ++e)                                                  \
        if (!used[L[e].i] && !used[L[e].j]) {                                                     \
            used[L[e].i] = used[L[e].j] = 1;                                                      \
            pi[np] = L[e].i; pj[np] = L[e].j; ++np;                                               \
        }                                                                                         \
    free(L); free(used);                                                                          \
    return np;                                                                                    \
}                                                                                                 \
static R SFX(colsq)(const R *G, int n, int skip_diag)                                             \
{                                                                                                 \
    R tot = 0;                                                                                    \
    for (int c = 0; c < n; ++c) {                                                                 \
        R sc = 0;                                                                                 \
        for (int r = 0; r < n; ++r)                                                               \
            if (!skip_diag || r != c) sc = FMA(G[(size_t)c * n + r], G[(size_t)c * n + r], sc);   \
        tot = tot + sc;                                                                           \
    }                                                                                             \
    return SQRT(tot);                                                                             \
}                                                                                                 \
static void SFX(rot)(R *x, R *y, const R m[4])                                                    \
{                                                                                                 \
    R a = *x, b = *y;                                                                             \
    *x = FMA(m[1], b, m[0] * a);                                                                  \
    *y = FMA(m[3], b, m[2] * a);                                                                  \
}                                                                                                 \
static int SFX(kogbet_impl)(int32_t n, const R *A, R *U, R *V, R *S, int max_sweeps,              \
                            double tol_factor, int32_t *sweeps, int32_t *info, int dyn)           \
{                                                                                                 \
    if (n < 1) return -1;                                                                         \
    size_t nn = (size_t)n * n;                                                                    \
    R *G = (R *)malloc(nn * sizeof(R));                                                           \
    int *pi = (int *)malloc(sizeof(int) * (size_t)n), *pj = (int *)malloc(sizeof(int) * (size_t)n); \
    R *pu = (R *)malloc(sizeof(R) * 4 * (size_t)n), *pv = (R *)malloc(sizeof(R) * 4 * (size_t)n);  \
    R *ps = (R *)malloc(sizeof(R) * 2 * (size_t)n);                                               \
    int *perm = (int *)malloc(sizeof(int) * (size_t)n);                                           \
    int finite = 1;                                                                               \
    for (size_t q = 0; q < nn; ++q) if (!isfinite(A[q])) finite = 0;                              \
    if (!finite) {                 /* non-finite input: NaN outputs, info -1 */                   \
        for (size_t q = 0; q < nn; ++q) { U[q] = NAN; V[q] = NAN; }                               \
        for (int q = 0; q < n; ++q) S[q] = NAN;                                                   \
        *sweeps = 0; *info = -1;                                                                  \
        free(G); free(pi); free(pj); free(pu); free(pv); free(ps); free(perm);                    \
        return 0;                                                                                 \
    }                                                                                             \
    memcpy(G, A, nn * sizeof(R));                                                                 \
    for (size_t q = 0; q < nn; ++q) { U[q] = 0; V[q] = 0; }                                       \
    for (int q = 0; q < n; ++q) { U[(size_t)q * n + q] = 1; V[(size_t)q * n + q] = 1; }           \
    int emax = INT32_MIN;                                                                         \
    for (size_t q = 0; q < nn; ++q) if (G[q] != 0) { int e = ILOGB(G[q]); if (e > emax) emax = e; } \
    int k = (emax == INT32_MIN) ? 0 : -(emax + 1);                                                \
    for (size_t q = 0; q < nn; ++q) G[q] = SCALBN(G[q], k);                                       \
    R tol = (R)tol_factor * (R)n * EPS * SFX(colsq)(G, n, 0);                                     \
    int sw = 0;                                                                                   \
    R off = SFX(colsq)(G, n, 1);                                                                  \
    while (!(off < tol) && sw < max_sweeps && off > 0) {                                          \
        for (int st = 0; st < n; ++st) {                                                          \
            int np = 0;                                                                           \
            if (dyn) np = SFX(k2ref_dyn_pairs)(n, G, pi, pj);                                     \
            else                                                                                  \
                for (int i = 0; i < n; ++i) {                                                     \
                    int j = (st - i + n) % n;                                                     \
                    if (i < j) { pi[np] = i; pj[np] = j; ++np; }                                  \
                }                                                                                 \
            for (int p = 0; p < np; ++p) {                                                        \
                int i = pi[p], j = pj[p];                                                         \
                PIVOT(G[(size_t)i * n + i], G[(size_t)i * n + j], G[(size_t)j * n + i],           \
                      G[(size_t)j * n + j], &pu[4 * p], &pv[4 * p], &ps[2 * p]);                  \
            }                                                                                     \
            for (int p = 0; p < np; ++p)                   /* rows i, j: U-hat^T */               \
                for (int c = 0; c < n; ++c)                                                       \
                    SFX(rot)(&G[(size_t)c * n + pi[p]], &G[(size_t)c * n + pj[p]], &pu[4 * p]);   \
            for (int p = 0; p < np; ++p)                   /* columns i, j: V-hat */              \
                for (int r = 0; r < n; ++r)                                                       \
                    SFX(rot)(&G[(size_t)pi[p] * n + r], &G[(size_t)pj[p] * n + r], &pv[4 * p]);   \
            for (int p = 0; p < np; ++p)                                                          \
                for (int r = 0; r < n; ++r) {                                                     \
                    SFX(rot)(&U[(size_t)pi[p] * n + r], &U[(size_t)pj[p] * n + r], &pu[4 * p]);   \
                    SFX(rot)(&V[(size_t)pi[p] * n + r], &V[(size_t)pj[p] * n + r], &pv[4 * p]);   \
                }                                                                                 \
            for (int p = 0; p < np; ++p) {                                                        \
                int i = pi[p], j = pj[p];                                                         \
                G[(size_t)i * n + i] = ps[2 * p];                                                 \
                G[(size_t)j * n + j] = ps[2 * p + 1];                                             \
                G[(size_t)j * n + i] = 0;                                                         \
                G[(size_t)i * n + j] = 0;                                                         \
            }                                                                                     \
        }                                                                                         \
        ++sw;                                                                                     \
        off = SFX(colsq)(G, n, 1);                                                                \
    }                                                                                             \
    *sweeps = sw;                                                                                 \
    *info = (off < tol || off == 0) ? 0 : 1;                                                      \
    /* a negative diagonal element (left by an early exit) gives its sign to U's column */    \
    for (int q = 0; q < n; ++q)                                                                   \
        if (G[(size_t)q * n + q] < 0) {                                                           \
            G[(size_t)q * n + q] = -G[(size_t)q * n + q];                                         \
            for (int r = 0; r < n; ++r) U[(size_t)q * n + r] = -U[(size_t)q * n + r];             \
        }                                                                                         \
    /* stable sort of the diagonal into descending order */                                      \
    for (int q = 0; q < n; ++q) perm[q] = q;                                                      \
    for (int a = 1; a < n; ++a) {                                                                 \
        int x = perm[a], b = a - 1;                                                               \
        while (b >= 0 && G[(size_t)perm[b] * n + perm[b]] < G[(size_t)x * n + x]) {              \
            perm[b + 1] = perm[b]; --b;                                                           \
        }                                                                                         \
        perm[b + 1] = x;                                                                          \
    }                                                                                             \
    R *T = (R *)malloc(nn * sizeof(R));                                                           \
    for (int q = 0; q < n; ++q) S[q] = SCALBN(G[(size_t)perm[q] * n + perm[q]], -k);              \
    memcpy(T, U, nn * sizeof(R));                                                                 \
    for (int q = 0; q < n; ++q) memcpy(&U[(size_t)q * n], &T[(size_t)perm[q] * n], sizeof(R) * (size_t)n); \
    memcpy(T, V, nn * sizeof(R));                                                                 \
    for (int q = 0; q < n; ++q) memcpy(&V[(size_t)q * n], &T[(size_t)perm[q] * n], sizeof(R) * (size_t)n); \
    free(T); free(G); free(pi); free(pj); free(pu); free(pv); free(ps); free(perm);               \
    return 0;                                                                                     \
}                                                                                                 \
int SFX(k2ref_kogbet)(int32_t n, const R *A, R *U, R *V, R *S, int max_sweeps, double tol_factor, \
                      int32_t *sweeps, int32_t *info)                                             \
{                                                                                                 \
    return SFX(kogbet_impl)(n, A, U, V, S, max_sweeps, tol_factor, sweeps, info, 0);              \
}                                                                                                 \
int SFX(k2ref_kogbet_dyn)(int32_t n, const R *A, R *U, R *V, R *S, int max_sweeps,                \
                          double tol_factor, int32_t *sweeps, int32_t *info)                      \
{                                                                                                 \
    return SFX(kogbet_impl)(n, A, U, V, S, max_sweeps, tol_factor, sweeps, info, 1);              \
}

/* dA = U diag(dS) V^T: element (r, c) accumulates (U_rq dS_q) V_cq over q = 0..n-1 with fma. */
#define SIGBWD_BODY(R, SFX, FMA)                                                                  \
void SFX(k2ref_kog_sigma_bwd)(int32_t n, const R *U, const R *V, const R *dS, R *dA)             \
{                                                                                                 \
    for (int c = 0; c < n; ++c)                                                                   \
        for (int r = 0; r < n; ++r) {                                                             \
            R acc = 0;                                                                            \
            for (int q = 0; q < n; ++q)                                                           \
                acc = FMA(U[(size_t)q * n + r] * dS[q], V[(size_t)q * n + c], acc);               \
            dA[(size_t)c * n + r] = acc;                                                          \
        }                                                                                         \
}

#define SFXD(x) x##_d
#define SFXS(x) x##_s
KOG_BODY(double, SFXD, k2ref_pivot_d, fma, sqrt, scalbn, ilogb, 0x1p-52)
KOG_BODY(float, SFXS, k2ref_pivot_s, fmaf, sqrtf, scalbnf, ilogbf, 0x1p-23f)
SIGBWD_BODY(double, SFXD, fma)
SIGBWD_BODY(float, SFXS, fmaf)
