/*
 * Oracle of the SVD of a rectangular matrix by preprocessing to a square one (Sect. 1: an
 * m x n matrix, m > n, is first reduced by a URV-type factorization such as the QR
 * factorization with column pivoting; for m < n the SVD of the transpose is computed),
 * followed by the n x n Kogbetliantz method of k2ref_kog.c.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper fixes neither the factorization's formulas nor their order; the readings taken
 * (also listed in the design notes), chosen so that every step is a fixed sequence of
 * correctly rounded operations:
 *  - B = A (m >= n) or A^T (m < n), p x q with p >= q; B is scaled by the power of two 2^k
 *    that brings its largest element into [1/2, 1) (exact; the singular values are scaled
 *    back by 2^-k);
 *  - Householder QR with column pivoting, B P = Q R: at step j the squared norms of the
 *    columns c >= j over rows j..p-1 are recomputed, each an fma accumulation in increasing
 *    row order starting from 0; the pivot is the first column with the largest squared norm;
 *    it is swapped with column j; with x = B[j:p, j], ||x|| = sqrt(its squared norm),
 *    alpha = -sign(x0) ||x|| (sign(+-0) = +1), v = x with v0 = x0 - alpha, and
 *    v^T v = 2 (||x|| (||x|| + |x0|)); every column c > j gets s = v0 B[j][c] followed by
 *    fma(v_i, B[j+i][c], s) in increasing i, f = (s + s) / v^T v, then
 *    B[j+i][c] = fma(-f, v_i, B[j+i][c]); B[j][j] = alpha, zeros below; a zero x is left
 *    alone (no reflector);
 *  - Q (p x q) = H_0 ... H_{q-1} [I; 0], the reflectors applied to the columns of [I; 0] in
 *    the order q-1, ..., 0 with the same formulas; R = the upper triangle of B (q x q);
 *  - R = U_R diag(sigma) V_R^T by the Kogbetliantz oracle; B = (Q U_R) diag(sigma) (P V_R)^T,
 *    each element of Q U_R an fma accumulation over k in increasing order starting from
 *    the product of the first terms; P V_R moves row j of V_R to row perm[j];
 *  - m >= n: U = Q U_R (m x n), V = P V_R (n x n); m < n: U = P V_R (m x m), V = Q U_R
 *    (n x m); sigma (min(m, n)) descending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int k2ref_kogbet_d(int32_t n, const double *A, double *U, double *V, double *S, int max_sweeps, double tol_factor,
                   int32_t *sweeps, int32_t *info);
int k2ref_kogbet_s(int32_t n, const float *A, float *U, float *V, float *S, int max_sweeps, double tol_factor,
                   int32_t *sweeps, int32_t *info);

#define RECT_BODY(R, SFX, KOGBET, FMA, SQRT, SCALBN, ILOGB, FABS)                                      \
int SFX(k2ref_gesvdr)(int32_t m, int32_t n, const R *A, R *U, R *V, R *S, int max_sweeps,             \
                      double tol_factor, int32_t *sweeps, int32_t *info)                              \
{                                                                                                     \
    if (m < 1 || n < 1) return -1;                                                                    \
    const int tr = m < n;                                                                             \
    const int p = tr ? n : m, q = tr ? m : n;                                                         \
    R *B = (R *)malloc(sizeof(R) * (size_t)p * q);                                                    \
    R *Q = (R *)malloc(sizeof(R) * (size_t)p * q);                                                    \
    R *Rm = (R *)malloc(sizeof(R) * (size_t)q * q);                                                   \
    R *UR = (R *)malloc(sizeof(R) * (size_t)q * q), *VR = (R *)malloc(sizeof(R) * (size_t)q * q);      \
    R *vv = (R *)malloc(sizeof(R) * (size_t)q), *nrm = (R *)malloc(sizeof(R) * (size_t)q);             \
    R *alph = (R *)malloc(sizeof(R) * (size_t)q);                                                     \
    int *perm = (int *)malloc(sizeof(int) * (size_t)q);                                               \
    int finite = 1, emax = INT32_MIN;                                                                 \
    for (int c = 0; c < q; ++c)                                                                       \
        for (int r = 0; r < p; ++r) {                                                                 \
            R x = tr ? A[(size_t)r * m + c] : A[(size_t)c * m + r];      /* B = A or A^T */          \
            B[(size_t)c * p + r] = x;                                                                 \
            if (!isfinite(x)) finite = 0;                                                             \
            else if (x != 0) { int e = ILOGB(x); if (e > emax) emax = e; }                            \
        }                                                                                             \
    if (!finite) {                                                                                    \
        for (size_t e = 0; e < (size_t)m * q; ++e) U[e] = NAN;                                        \
        for (size_t e = 0; e < (size_t)n * q; ++e) V[e] = NAN;                                        \
        for (int e = 0; e < q; ++e) S[e] = NAN;                                                       \
        *sweeps = 0; *info = -1;                                                                      \
        free(B); free(Q); free(Rm); free(UR); free(VR); free(vv); free(nrm); free(alph); free(perm);              \
        return 0;                                                                                     \
    }                                                                                                 \
    const int k = (emax == INT32_MIN) ? 0 : -(emax + 1);                                              \
    for (size_t e = 0; e < (size_t)p * q; ++e) B[e] = SCALBN(B[e], k);                                \
    for (int c = 0; c < q; ++c) perm[c] = c;                                                          \
    for (int j = 0; j < q; ++j) {                                                                     \
        for (int c = j; c < q; ++c) {                                                                 \
            R sq = 0;                                                                                 \
            for (int r = j; r < p; ++r) sq = FMA(B[(size_t)c * p + r], B[(size_t)c * p + r], sq);     \
            nrm[c] = sq;                                                                              \
        }                                                                                             \
        int piv = j;                                                                                  \
        for (int c = j + 1; c < q; ++c) if (nrm[c] > nrm[piv]) piv = c;                               \
        if (piv != j) {                                                                               \
            for (int r = 0; r < p; ++r) {                                                             \
                R t = B[(size_t)j * p + r]; B[(size_t)j * p + r] = B[(size_t)piv * p + r]; B[(size_t)piv * p + r] = t; \
            }                                                                                         \
            int t = perm[j]; perm[j] = perm[piv]; perm[piv] = t;                                      \
        }                                                                                             \
        R *x = B + (size_t)j * p + j;                                                                 \
        const int L = p - j;                                                                          \
        if (nrm[piv] == 0) { vv[j] = 0; alph[j] = x[0]; continue; }    /* no reflector */            \
        const R nx = SQRT(nrm[piv]);                                                                  \
        const R x0 = x[0];                                                                            \
        const R alpha = (x0 < 0) ? nx : -nx;                                                          \
        alph[j] = alpha;                                                                              \
        vv[j] = 2 * (nx * (nx + FABS(x0)));                                                           \
        x[0] = x0 - alpha;                              /* v: x[0] = v0, x[i] = v_i below */          \
        for (int c = j + 1; c < q; ++c) {                                                             \
            R *y = B + (size_t)c * p + j;                                                             \
            R s = x[0] * y[0];                                                                        \
            for (int i = 1; i < L; ++i) s = FMA(x[i], y[i], s);                                       \
            const R f = (s + s) / vv[j];                                                              \
            for (int i = 0; i < L; ++i) y[i] = FMA(-f, x[i], y[i]);                                   \
        }                                                                                             \
    }                                                                                                 \
    /* R: the strict upper triangle of B and the alphas on the diagonal */                           \
    for (int c = 0; c < q; ++c)                                                                       \
        for (int r = 0; r < q; ++r)                                                                   \
            Rm[(size_t)c * q + r] = (r < c) ? B[(size_t)c * p + r] : (r == c ? alph[c] : 0);          \
    /* Q = H_0 ... H_{q-1} [I; 0] */                                                                  \
    for (size_t e = 0; e < (size_t)p * q; ++e) Q[e] = 0;                                              \
    for (int c = 0; c < q; ++c) Q[(size_t)c * p + c] = 1;                                             \
    for (int j = q - 1; j >= 0; --j) {                                                                \
        if (vv[j] == 0) continue;                                                                     \
        const R *x = B + (size_t)j * p + j;                                                           \
        const int L = p - j;                                                                          \
        for (int c = 0; c < q; ++c) {                                                                 \
            R *y = Q + (size_t)c * p + j;                                                             \
            R s = x[0] * y[0];                                                                        \
            for (int i = 1; i < L; ++i) s = FMA(x[i], y[i], s);                                       \
            const R f = (s + s) / vv[j];                                                              \
            for (int i = 0; i < L; ++i) y[i] = FMA(-f, x[i], y[i]);                                   \
        }                                                                                             \
    }                                                                                                 \
    int rc = KOGBET(q, Rm, UR, VR, S, max_sweeps, tol_factor, sweeps, info);                          \
    if (rc == 0) {                                                                                    \
        for (int e = 0; e < q; ++e) S[e] = SCALBN(S[e], -k);                                          \
        R *QU = tr ? V : U;                             /* Q U_R: p x q */                            \
        R *PV = tr ? U : V;                             /* P V_R: q x q */                            \
        for (int c = 0; c < q; ++c)                                                                   \
            for (int r = 0; r < p; ++r) {                                                             \
                R acc = Q[r] * UR[(size_t)c * q];                                                     \
                for (int t = 1; t < q; ++t) acc = FMA(Q[(size_t)t * p + r], UR[(size_t)c * q + t], acc); \
                QU[(size_t)c * p + r] = acc;                                                          \
            }                                                                                         \
        for (int c = 0; c < q; ++c)                                                                   \
            for (int j = 0; j < q; ++j) PV[(size_t)c * q + perm[j]] = VR[(size_t)c * q + j];          \
    }                                                                                                 \
    free(B); free(Q); free(Rm); free(UR); free(VR); free(vv); free(nrm); free(alph); free(perm);                  \
    return rc;                                                                                        \
}

#define SFXD(x) x##_d
#define SFXS(x) x##_s
RECT_BODY(double, SFXD, k2ref_kogbet_d, fma, sqrt, scalbn, ilogb, fabs)
RECT_BODY(float, SFXS, k2ref_kogbet_s, fmaf, sqrtf, scalbnf, ilogbf, fabsf)
