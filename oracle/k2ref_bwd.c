/*
 * Oracle of the backward (adjoint) of the batched 2x2 SVD, TEST INFRASTRUCTURE ONLY.
 *
 * The paper has no backward.  This is the textbook adjoint of a square real SVD
 * G = U S V^T with distinct singular values (the perturbation of U and V is a rotation
 * whose angle follows from keeping U^T dG V diagonal), evaluated in binary128:
 *   J = U^T dU, K = V^T dV,
 *   F12 = -1 / (g (s1 + s2)), g = max(s1 - s2, tau s1), F21 = -F12, F12 = 0 when s1 = 0,
 *   M = diag(dS) + (F o (J - J^T)) S + S (F o (K - K^T)),
 *   dG = U M V^T.
 * Pinned by central finite differences of the oracle's forward (tests).
 */
#include <stdint.h>

typedef _Float128 qb_t;

/* planes with leading dimension ld: U, V, dU, dV, dG in column-major 4 planes; S, dS 2 planes.
 * dS, dU, dV may be NULL (zero). */
int k2ref_gesvd2_bwd_d(int64_t n, const double *U, const double *S, const double *V, int64_t ld,
                       const double *dS, const double *dU, const double *dV, double *dG, double tau)
{
    if (n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        qb_t u[2][2] = { { U[i], U[2 * ld + i] }, { U[ld + i], U[3 * ld + i] } };
        qb_t v[2][2] = { { V[i], V[2 * ld + i] }, { V[ld + i], V[3 * ld + i] } };
        qb_t du[2][2] = { { 0, 0 }, { 0, 0 } }, dv[2][2] = { { 0, 0 }, { 0, 0 } };
        if (dU) { du[0][0] = dU[i]; du[1][0] = dU[ld + i]; du[0][1] = dU[2 * ld + i]; du[1][1] = dU[3 * ld + i]; }
        if (dV) { dv[0][0] = dV[i]; dv[1][0] = dV[ld + i]; dv[0][1] = dV[2 * ld + i]; dv[1][1] = dV[3 * ld + i]; }
        qb_t s1 = S[i], s2 = S[ld + i];
        qb_t d1 = dS ? dS[i] : 0, d2 = dS ? dS[ld + i] : 0;
        /* J = U^T dU, K = V^T dV */
        qb_t J[2][2], K[2][2];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                J[p][q] = u[0][p] * du[0][q] + u[1][p] * du[1][q];
                K[p][q] = v[0][p] * dv[0][q] + v[1][p] * dv[1][q];
            }
        qb_t F12 = 0;
        if (s1 > 0) {
            qb_t g = s1 - s2;
            if (g < (qb_t)tau * s1) g = (qb_t)tau * s1;
            F12 = -1 / (g * (s1 + s2));
        }
        qb_t F21 = -F12;
        qb_t sg[2] = { s1, s2 };
        qb_t M[2][2];
        M[0][0] = d1;
        M[1][1] = d2;
        M[0][1] = F12 * (J[0][1] - J[1][0]) * sg[1] + sg[0] * F12 * (K[0][1] - K[1][0]);
        M[1][0] = F21 * (J[1][0] - J[0][1]) * sg[0] + sg[1] * F21 * (K[1][0] - K[0][1]);
        /* dG = U M V^T */
        qb_t W[2][2], D[2][2];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q)
                W[p][q] = u[p][0] * M[0][q] + u[p][1] * M[1][q];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q)
                D[p][q] = W[p][0] * v[q][0] + W[p][1] * v[q][1];
        dG[i] = (double)D[0][0];
        dG[ld + i] = (double)D[1][0];
        dG[2 * ld + i] = (double)D[0][1];
        dG[3 * ld + i] = (double)D[1][1];
    }
    return 0;
}
