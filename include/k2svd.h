/*
 * libk2svd -- batched SVD of real 2x2 matrices by the enhanced Kogbetliantz method
 * (V. Novakovic, "Arithmetical enhancements of the Kogbetliantz method for the SVD of
 * order two", arXiv 2407.13116), on NVIDIA GB300 (sm_103a).
 *
 * Problem (Sect. 1): G = U Sigma V^T with U, V orthogonal and sigma1 >= sigma2 >= 0.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Pointers.  Every array argument is a DEVICE pointer (cudaMalloc'd or managed
 *   memory), owned by the caller; the library never allocates, frees or keeps them.
 *   Optional arrays are marked "nullable" and are skipped when NULL.
 * Library memory.  No entry point allocates device memory; scratch, where an entry point
 *   needs it, is a caller-supplied workspace (k2svd_dkogbet_noalloc: a static array).
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls are asynchronous and stream-ordered; a return value of 0 means
 *   the work was enqueued.  Kernel faults surface as CUDA errors on that stream.
 * SoA planes.  A "k-plane array" X of leading dimension ld >= batch holds element
 *   (plane j, matrix i) at X[j*ld + i].  2x2 matrices use 4 planes in column-major
 *   element order (x11, x21, x12, x22); singular values use 2 planes (sigma1, sigma2).
 * Precision.  The d-variants compute in IEEE binary64 with binary128 emulated
 *   exactly where eq. (EXT) of Sect. 3.2.2 asks for a wider type; the s-variants in
 *   binary32 with binary64 for eq. (EXT).  Every result is bitwise reproducible and
 *   independent of the launch configuration (end of Sect. 3.3.2).
 * Errors.  Return 0 on success; -i when argument i (1-based) is invalid, checked in
 *   order, LAPACK style; K2SVD_ECUDA when a CUDA call failed (the CUDA error is left
 *   for cudaGetLastError to report).  Per-matrix conditions go to `info` (below).
 * Graph capture.  The 2x2 entry points (k2svd_?gesvd2, k2svd_?trsvd2 and their variants,
 *   k2svd_?gesvd2_bwd, k2svd_?prescale2, k2svd_?lasv2, k2svd_?gesvd2 of complex type) only
 *   launch kernels on device pointers and may be captured into a CUDA graph.  The n x n
 *   entry points (k2svd_?kogbet, k2svd_dkogbet_noalloc, k2svd_?kog_sigma_bwd,
 *   k2svd_?gesvdr) copy a host-side table of the call to the device; a captured copy would
 *   read that table at replay time, after it is gone, so they return K2SVD_ECAPTURE on a
 *   stream that is being captured (K2SVD_KOG_GRAPH builds and caches a graph internally
 *   instead).
 * Inputs must be finite (Sect. 2).  A matrix with a NaN or infinite element gets
 *   info = -1 and NaN in all its outputs; the other matrices are unaffected.
 */
#ifndef K2SVD_H
#define K2SVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define K2SVD_ECUDA (-1000)
#define K2SVD_ECAPTURE (-1002)   /* the stream is being captured into a CUDA graph */

/* info bits per matrix (when info != NULL and the input is finite):
 *   bits 0-3  zero-pattern type t of G (eq. (ts): 1 = g11, 2 = g21, 4 = g12, 8 = g22 non-zero)
 *   bits 4-7  type t' after the prescaling (Sect. 3.1)
 *   bits 8-15 branch flags: */
#define K2SVD_INFO_EXT      (1 << 8)   /* one element of R by eq. (EXT) (Sect. 3.2.2)          */
#define K2SVD_INFO_FALLBACK (1 << 9)   /* t'=15 with r12''=0 or r22''=0, finished as Sect. 3.1 */
#define K2SVD_INFO_SWAP     (1 << 10)  /* r11 < r22: transpose-swap of eq. (RT)                */
#define K2SVD_INFO_T2F2     (1 << 11)  /* tan(2 phi) by eq. (t2f'')                            */
#define K2SVD_INFO_T2F3     (1 << 12)  /* tan(2 phi) by eq. (t2f''')                           */
#define K2SVD_INFO_T2INF    (1 << 13)  /* tan(2 phi) = inf, tan(phi) = 1 (Alg. 1)              */
#define K2SVD_INFO_TPINF    (1 << 14)  /* tan(psi) = inf, eq. (tp') (Alg. 2)                   */
#define K2SVD_INFO_PSIG     (1 << 15)  /* singular values reordered by eq. (prec) (Alg. 2)     */
#define K2SVD_INFO_T2NCR    (1 << 18)  /* tan(2 phi) by Alg. 1's branch for a hypot that is not
                                          correctly rounded (the k2svd_?gesvd2_ncr variant only) */

/*
 * k2svd_dgesvd2 / k2svd_sgesvd2 -- SVD of `batch` general real 2x2 matrices.
 * Method: Sect. 3 phases 1-3: the prescaling of eqs. (eG), (s), (ts); the simple cases
 * of Sect. 3.1; the URV factorization of Sect. 3.2 (eq. (QR15), (EXT)); the SVD of the
 * triangular factor by Alg. 1 and Alg. 2 with a correctly rounded hypot; the left-vector
 * heuristic of Sect. 3.3.2 (eqs. (p+t), (p-t), (tan+-), (UV)).
 *
 *   batch   number of matrices, >= 0 (0: nothing is launched)
 *   G       4-plane input, ld = ldg (read only)
 *   U, V    4-plane outputs (ld = ldu, ldv): G = U diag(S) V^T, U and V exactly
 *           representable products of signed permutations and rotations, never Inf/NaN
 *   S       2-plane output (ld = lds): sigma1 >= sigma2 >= 0 rounded once to the working
 *           type (they may overflow to +Inf or underflow; see Se/Sf)
 *   Se, Sf  nullable 2-plane outputs (ld = lds): the exact exponent-"mantissa" form
 *           sigma_i = Sf_i * 2^Se_i with 1 <= Sf_i < 2 (or Sf_i = 0, Se_i = 0), which
 *           never overflows or underflows (Sect. 3.3.2)
 *   info    nullable, one int32 per matrix (bits above)
 *   stream  cudaStream_t as void*
 * Planes of different arrays must not overlap.  Argument order for error codes:
 * 1 batch, 2 G, 3 ldg, 4 U, 5 ldu, 6 V, 7 ldv, 8 S, 9 lds.
 * k2svd_dgesvd2 on 65536 or more matrices runs the method as two kernels per chunk of the
 * batch (phases 1-2, then phase 3); between the two launches a matrix's intermediate state
 * (48 bytes) is kept in its own U, V and S output planes, so the call needs no scratch
 * memory.  The results are the same bits as the single fused kernel's.
 */
int k2svd_dgesvd2(int64_t batch, const double *G, int64_t ldg,
                  double *U, int64_t ldu, double *V, int64_t ldv,
                  double *S, int64_t lds, int32_t *Se, double *Sf,
                  int32_t *info, void *stream);
int k2svd_sgesvd2(int64_t batch, const float *G, int64_t ldg,
                  float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *Se, float *Sf,
                  int32_t *info, void *stream);

/*
 * k2svd_dtrsvd2 / k2svd_strsvd2 -- SVD of `batch` upper-triangular matrices
 * R = [[F, Gu], [0, H]] given as three planes (the xLASV2 argument shape, Sect. 1 and the
 * remark before the three-phase outline of Sect. 3).  Any signs and zeros are allowed;
 * the result equals k2svd_?gesvd2 on [[F, Gu], [0, H]] bit for bit, and phase 2 of
 * Sect. 3.2.2 (the t'=15 URV) never runs.  Unlike xLASV2 the singular values are
 * non-negative and the full U, V are returned.
 * Argument order for error codes: 1 batch, 2 F, 3 Gu, 4 H, 5 U, 6 ldu, 7 V, 8 ldv, 9 S, 10 lds.
 */
int k2svd_dtrsvd2(int64_t batch, const double *F, const double *Gu, const double *H,
                  double *U, int64_t ldu, double *V, int64_t ldv,
                  double *S, int64_t lds, int32_t *Se, double *Sf,
                  int32_t *info, void *stream);
int k2svd_strsvd2(int64_t batch, const float *F, const float *Gu, const float *H,
                  float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *Se, float *Sf,
                  int32_t *info, void *stream);

/*
 * k2svd_dgesvd2_ncr / k2svd_sgesvd2_ncr, k2svd_dtrsvd2_ncr / k2svd_strsvd2_ncr -- the same
 * SVDs with a hypot that is not correctly rounded, the case for which Alg. 1 (Sect. 3.3.1)
 * has its own branch: after the three special cases of Alg. 1, tan(2 phi) comes from
 * x = r12/r11, y = r22/r11 (r11 > r12) or x = r11/r12, y = r22/r12 (otherwise) as
 * fl(fl(2x)y) or 2y divided by max(fma(x - y, x + y, 1), 0), without squaring; and every
 * hypot of the method (Alg. 1, Alg. 2, Sect. 3.1, Sect. 3.2.2) is xLAPY2's scaled formula
 * w * sqrt(fma(q, q, 1)), q = z / w, w = max(|x|,|y|), z = min(|x|,|y|), each step rounded to
 * nearest (at most 3.5 units of 2^-p from the exact value).  The paper gives no relative
 * error bound for this variant.  Arguments, layout, ownership, error codes and the handling
 * of non-finite inputs are those of k2svd_?gesvd2 and k2svd_?trsvd2; info carries
 * K2SVD_INFO_T2NCR where the branch ran.
 */
int k2svd_dgesvd2_ncr(int64_t batch, const double *G, int64_t ldg,
                      double *U, int64_t ldu, double *V, int64_t ldv,
                      double *S, int64_t lds, int32_t *Se, double *Sf,
                      int32_t *info, void *stream);
int k2svd_sgesvd2_ncr(int64_t batch, const float *G, int64_t ldg,
                      float *U, int64_t ldu, float *V, int64_t ldv,
                      float *S, int64_t lds, int32_t *Se, float *Sf,
                      int32_t *info, void *stream);
int k2svd_dtrsvd2_ncr(int64_t batch, const double *F, const double *Gu, const double *H,
                      double *U, int64_t ldu, double *V, int64_t ldv,
                      double *S, int64_t lds, int32_t *Se, double *Sf,
                      int32_t *info, void *stream);
int k2svd_strsvd2_ncr(int64_t batch, const float *F, const float *Gu, const float *H,
                      float *U, int64_t ldu, float *V, int64_t ldv,
                      float *S, int64_t lds, int32_t *Se, float *Sf,
                      int32_t *info, void *stream);

/*
 * k2svd_dgesvdr_ws / k2svd_sgesvdr_ws, k2svd_dgesvdr / k2svd_sgesvdr -- SVD of `batch`
 * rectangular matrices of uneven shapes, A_i = U_i diag(S_i) V_i^T with k = min(m, n)
 * singular values (Sect. 1: an m x n matrix, m > n, is first reduced to a square one by a
 * URV-type factorization such as QR with column pivoting; for m < n the transpose is
 * decomposed).  B = A (or A^T), p x q with p >= q, is scaled by the power of two that puts
 * its largest element in [1/2, 1); Householder QR with column pivoting B P = Q R (squared
 * column norms recomputed at every step by fma in increasing row order, the first column of
 * largest norm as pivot, alpha = -sign(x0) ||x||, v0 = x0 - alpha,
 * v^T v = 2 ||x|| (||x|| + |x0|), each column updated with f = (s + s) / v^T v); R (q x q)
 * goes through the n x n Kogbetliantz driver (k2svd_?kogbet, same max_sweeps, tol_factor
 * and sweeps/info semantics); U = Q U_R, V = P V_R (exchanged for m < n).  Results are
 * bitwise reproducible.  The paper's "dynamic ordering" of pivots is not implemented (the
 * square driver uses the modulus strategy).
 *
 *   batch            number of matrices, >= 0
 *   m, n             HOST arrays of the shapes, 1 <= m, n <= 65536, min(m, n) <= 4096
 *   aoffs            HOST array: A_i (m x n, column-major) starts at element aoffs[i] of A
 *   uoffs, voffs     HOST arrays: U_i (m x k) and V_i (n x k), column-major, in U and V
 *   soffs            HOST array: the k singular values of matrix i, descending, in S
 *   sweeps, info     nullable device arrays (one int32 per matrix), as for k2svd_?kogbet;
 *                    info -1 (NaN outputs) for a matrix with a non-finite element
 *   flags            0 or K2SVD_KOG_NOTUNE
 *   workspace        device scratch of ws_bytes bytes, 256-byte aligned, from
 *                    k2svd_?gesvdr_ws for the same batch, m, n and flags; owned by the caller
 * Argument order for error codes: 1 batch, 2 m, 3 n, 4 aoffs, 5 uoffs, 6 voffs, 7 soffs,
 * 8 A, 9 U, 10 V, 11 S, 14 max_sweeps, 15 tol_factor, 16 flags, 17 workspace, 18 ws_bytes;
 * -19 when the square driver rejects the reduced problem; K2SVD_ECUDA for CUDA errors;
 * K2SVD_ECAPTURE on a stream that is being captured into a CUDA graph.
 */
int k2svd_dgesvdr_ws(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, size_t *ws_bytes);
int k2svd_sgesvdr_ws(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, size_t *ws_bytes);
int k2svd_dgesvdr(int64_t batch, const int32_t *m, const int32_t *n, const int64_t *aoffs, const int64_t *uoffs,
                  const int64_t *voffs, const int64_t *soffs, const double *A, double *U, double *V, double *S,
                  int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream);
int k2svd_sgesvdr(int64_t batch, const int32_t *m, const int32_t *n, const int64_t *aoffs, const int64_t *uoffs,
                  const int64_t *voffs, const int64_t *soffs, const float *A, float *U, float *V, float *S,
                  int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream);

/*
 * k2svd_zgesvd2 / k2svd_cgesvd2 -- SVD of `batch` complex 2x2 matrices (Sect. 3.4),
 * G = U diag(sigma1, sigma2) V^H with U, V unitary and sigma1 >= sigma2 >= 0.  A real G
 * (every imaginary part zero) gets the real method (k2svd_?gesvd2's results, imaginary parts
 * zero); a purely imaginary G = iH the real method on H with U = i U_H.  Otherwise the
 * matrix is prescaled over every real and imaginary component with the scale type raised by
 * one; a matrix with at most three nonzero elements is made real by row and column phases
 * conj(z)/|z|; a matrix without zeros is reduced as in Sect. 3.2.2 with complex column
 * norms, row phases that make the first column real, the real rotation (no (EXT), item 3)
 * and phases that make r12 and r22 real; the real method then runs on the real matrix and
 * U, V are formed by real-complex products.  Complex product (a,b)(c,d) is
 * (fma(a,c,-(b d)), fma(a,d,b c)) and |z| the correctly rounded hypot, so results are
 * bitwise reproducible.
 *
 *   batch        number of matrices, >= 0
 *   G, ldg       8 planes: (re, im) of g11, g21, g12, g22; ldg >= batch
 *   U, ldu       8 planes, same layout; V, ldv likewise
 *   S, lds       2 planes: sigma1, sigma2
 *   info         nullable int32 plane: t | t' << 4 | flags << 8 (flags of the real method,
 *                plus 0x100 for a purely imaginary G and 0x200 for the complex reduction;
 *                an element is nonzero when either part is); -1 for non-finite input (NaN
 *                outputs for that matrix)
 * Argument order for error codes: 1 batch, 2 G, 3 ldg, 4 U, 5 ldu, 6 V, 7 ldv, 8 S, 9 lds.
 */
int k2svd_zgesvd2(int64_t batch, const double *G, int64_t ldg, double *U, int64_t ldu, double *V, int64_t ldv,
                  double *S, int64_t lds, int32_t *info, void *stream);
int k2svd_cgesvd2(int64_t batch, const float *G, int64_t ldg, float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *info, void *stream);

/*
 * k2svd_dprescale2 / k2svd_sprescale2 -- phase 1 of the method on its own (Sect. 3.1,
 * eqs. (eG), (s); the phases "can be used on their own", Sect. 5): for each matrix the type
 * t (bit k set when element k of (g11, g21, g12, g22) is nonzero), the exponent
 * s = e_nu - e_G - (scale type + extra), where e_G is the largest exponent of a nonzero
 * element and the scale type is 2 for matrices without zeros, else 1; matrices of class 9
 * (at most one nonzero per row and column) are not scaled (s = 0).  Gs = 2^s G, exact for
 * s >= 0 and one correct rounding per element otherwise; t' is the type of Gs.  extra = 1
 * leaves the margin Sect. 4 suggests before calling xLASV2 on small inputs.
 *
 *   batch    number of matrices, >= 0
 *   G, ldg   4-plane input (g11, g21, g12, g22), ldg >= batch
 *   Gs, ldgs 4-plane output, ldgs >= batch; may be G with the same leading dimension
 *   s        int32 plane: the exponent s of each matrix
 *   types    nullable int32 plane: t | t' << 4, or -1 for a matrix with a non-finite element
 *            (copied unchanged with s = 0)
 *   extra    0 .. 64
 * Argument order for error codes: 1 batch, 2 G, 3 ldg, 4 Gs, 5 ldgs, 6 s, 8 extra.
 */
int k2svd_dprescale2(int64_t batch, const double *G, int64_t ldg, double *Gs, int64_t ldgs, int32_t *s,
                     int32_t *types, int32_t extra, void *stream);
int k2svd_sprescale2(int64_t batch, const float *G, int64_t ldg, float *Gs, int64_t ldgs, int32_t *s,
                     int32_t *types, int32_t extra, void *stream);

/*
 * k2svd_dlasv2 / k2svd_slasv2 -- the argument shape of LAPACK's xLASV2 (the SVD of an upper
 * triangular 2x2 matrix, the case the paper compares against, Sects. 1 and 4), computed by
 * this method: for R = [[F, G], [0, H]],
 *     [ CSL  SNL ]  R  [ CSR  -SNR ]   =   [ SSMAX    0   ]
 *     [-SNL  CSL ]     [ SNR   CSR ]       [   0    SSMIN ]
 * with (CSL, SNL), (CSR, SNR) the first columns of the method's U and V (k2svd_?trsvd2),
 * SSMAX = sigma1 >= 0 and SSMIN = +-sigma2 carrying the sign of det R.  Every output is a
 * plane of `batch` elements (device pointers); a matrix with a non-finite input gets NaN
 * outputs.  The values differ from LAPACK's (a different method; LAPACK may also return a
 * negative SSMAX), the identity above holds for both.
 * Argument order for error codes: 1 batch, 2 F, 3 G, 4 H, 5 ssmin, 6 ssmax, 7 snr, 8 csr,
 * 9 snl, 10 csl.
 */
int k2svd_dlasv2(int64_t batch, const double *F, const double *G, const double *H, double *ssmin, double *ssmax,
                 double *snr, double *csr, double *snl, double *csl, void *stream);
int k2svd_slasv2(int64_t batch, const float *F, const float *G, const float *H, float *ssmin, float *ssmax,
                 float *snr, float *csr, float *snl, float *csl, void *stream);

/*
 * k2svd_dgesvd2_bwd / k2svd_sgesvd2_bwd -- adjoint (backward) of the batched 2x2 SVD.
 * The paper has no backward; this is the standard adjoint of a square SVD G = U S V^T
 * with distinct singular values, with a gap threshold for near-equal ones:
 *   J = U^T dU, K = V^T dV, a = J12 - J21, b = K12 - K21,
 *   F12 = -1 / (max(s1 - s2, gap_rtol * s1) * (s1 + s2))  (F12 = 0 when s1 = 0),
 *   M = [[dS1, F12 (a s2 + b s1)], [F12 (a s1 + b s2), dS2]],   dG = U M V^T.
 * It is evaluated after scaling s1, s2 by the power of two that brings s1 into [1, 2),
 * so that no intermediate overflows or underflows for any representable s1 > 0.
 *
 *   batch    number of matrices, >= 0
 *   U, V     4-plane outputs of k2svd_?gesvd2 (read only)
 *   S        2-plane singular values of k2svd_?gesvd2 (read only)
 *   ld       leading dimension of every plane array of this call, >= batch
 *   dS       nullable 2-plane upstream gradient of S (NULL = zero)
 *   dU, dV   nullable 4-plane upstream gradients of U and V (NULL = zero)
 *   dG       4-plane output, the gradient with respect to G (column-major planes)
 *   gap_rtol relative gap threshold tau >= 0 (1e-10 is a good default); pairs with
 *            s1 - s2 < tau s1 use tau s1 in place of the gap
 *   stream   cudaStream_t as void*
 * Argument order for error codes: 1 batch, 2 U, 3 S, 4 V, 5 ld, 9 dG, 10 gap_rtol.
 * Non-finite inputs give non-finite outputs for that matrix only.
 */
int k2svd_dgesvd2_bwd(int64_t batch, const double *U, const double *S, const double *V, int64_t ld,
                      const double *dS, const double *dU, const double *dV, double *dG,
                      double gap_rtol, void *stream);
int k2svd_sgesvd2_bwd(int64_t batch, const float *U, const float *S, const float *V, int64_t ld,
                      const float *dS, const float *dU, const float *dV, float *dG,
                      float gap_rtol, void *stream);

/*
 * k2svd_dkogbet / k2svd_skogbet -- SVD of `batch` square matrices of uneven orders by the
 * parallel Kogbetliantz method, eq. (SVD) of Sect. 1: G_{k+1} = U_k^T G_k V_k with
 * U_{k+1} = U_k U_k-hat and V_{k+1} = V_k V_k-hat, where step k of a sweep transforms the
 * disjoint pivot pairs of the parallel modulus strategy (all pairs i < j with
 * i + j = k mod n, k = 0..n-1), each pivot [[g_ii, g_ij], [g_ji, g_jj]] decomposed by the
 * 2x2 method of Sect. 3.  Order of a step: all pivot SVDs from G_k, all row rotations, all
 * column rotations (U and V updated alike), then the pivot blocks set to diag(sigma1,
 * sigma2).  A rotated pair (x, y) becomes (fma(m21, y, m11 x), fma(m22, y, m12 x)).  G is
 * first scaled by the power of two that puts its largest element in [1/2, 1).  Sweeps stop
 * when off(G) < tol_factor * n * eps * ||G||_F (eps = 2^-52 / 2^-23; the norms summed
 * column by column in increasing index order) or after max_sweeps.  At exit a negative
 * diagonal element is negated with its column of U; the singular values are sorted into
 * descending order (stable), permuting U and V.  Results are bitwise
 * reproducible and independent of the launch configuration.
 *
 *   batch        number of matrices, >= 0
 *   n            HOST array of the orders, 1 <= n[i] <= 4096
 *   offs         HOST array: matrix i's A, U and V start at element offs[i] of their
 *                arrays, column-major with leading dimension n[i]
 *   soffs        HOST array: matrix i's singular values start at element soffs[i] of S
 *   A            input matrices (read only)
 *   U, V         outputs (may not alias A), A_i = U_i diag(S_i) V_i^T
 *   S            output singular values, descending, n[i] per matrix
 *   sweeps, info nullable device arrays (one int32 per matrix): sweeps performed; info 0 =
 *                converged, 1 = stopped at max_sweeps (the method never hangs)
 *   max_sweeps   >= 0; tol_factor > 0 (1.0: the bound above); the per-step form needs
 *                batch <= 65535
 *   flags        K2SVD_KOG_PLAIN: one launch per step (the per-step form, for comparison);
 *                K2SVD_KOG_GRAPH: capture the launches in a CUDA graph (cached for repeated
 *                calls with the same arguments) and launch the graph;
 *                K2SVD_KOG_NOTUNE: skip the block-size autotuner (defaults per order);
 *                K2SVD_KOG_DYNAMIC (experimental): the dynamic ordering instead of the
 *                modulus strategy (Sect. 1 names it as a candidate).  On a GB300 it needs
 *                about 18% fewer sweeps but runs about 4 times longer than the modulus
 *                strategy, since its pair selection cannot start before a step's rotations
 *                end; it is kept for studying the ordering.  The pairs of a step are taken greedily
 *                by decreasing weight w_ij = fma(g_ji, g_ji, g_ij^2) computed from G_k (ties:
 *                smaller i, then smaller j), each pair whose indices are both still free,
 *                up to floor(n/2) pairs; a sweep is still n steps.  Persistent form only
 *                (with K2SVD_KOG_PLAIN: error -13); the workspace grows by n(n-1)/2
 *                elements per matrix
 *   workspace    device scratch of ws_bytes bytes, 256-byte aligned, from k2svd_?kogbet_ws
 *                for the same batch, n and flags; owned by the caller, not kept after the call
 *                (a cached graph refers to it: keep it alive while reusing the same arguments)
 * Returns K2SVD_ECAPTURE when `stream` is being captured into a CUDA graph (the call copies
 * its host-side descriptor table; use K2SVD_KOG_GRAPH for a graph launch).
 * The persistent form groups the matrices by order into buckets; each bucket runs as one
 * persistent launch (one CTA per matrix at a time, longest first, G in shared memory up to
 * order 128 for double and 224 for float, else in the workspace), with the block size
 * picked per bucket by timing (first call per device).  The bucket launches run
 * concurrently on streams the library creates on a device's first call (one per bucket,
 * larger orders at higher priority, kept until exit), ordered after the work queued on
 * `stream` before the call and before the work queued on it after the call; with
 * K2SVD_KOG_GRAPH they are parallel branches of the cached graph.  Host threads may call
 * concurrently: the library's streams are used under a lock.  The host arrays are read
 * during the call only.  Argument order for error codes: 1 batch, 2 n, 3 offs, 4 soffs, 5 A, 6 U,
 * 7 V, 8 S, 11 max_sweeps, 12 tol_factor, 13 flags, 14 workspace, 15 ws_bytes.
 */
#define K2SVD_KOG_PLAIN  1
#define K2SVD_KOG_GRAPH  2
#define K2SVD_KOG_NOTUNE 4
#define K2SVD_KOG_DYNAMIC 8
int k2svd_dkogbet_ws(int64_t batch, const int32_t *n, int32_t flags, size_t *ws_bytes);
int k2svd_skogbet_ws(int64_t batch, const int32_t *n, int32_t flags, size_t *ws_bytes);
int k2svd_dkogbet(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs,
                  const double *A, double *U, double *V, double *S, int32_t *sweeps, int32_t *info,
                  int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream);
int k2svd_skogbet(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs,
                  const float *A, float *U, float *V, float *S, int32_t *sweeps, int32_t *info,
                  int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream);

/*
 * k2svd_dkogbet_noalloc -- k2svd_dkogbet for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a service entry point.  Some callers may not
 * allocate at all: a host whose device memory is entirely owned by another allocator (a
 * framework's caching allocator that reserved it up front), a path that must not fail on
 * an allocation, or a plugin that has no access to the allocator.  This entry needs no
 * workspace: its scratch (the work queues, the descriptor
 * table and, for orders above 128, the working copies of G) lives in one static device
 * array of K2SVD_KOG_NOALLOC_BYTES bytes that every GPU holds from the time it loads the
 * library until the process exits.  The call makes no device or host heap allocation.
 *   Arguments, results and conventions are those of k2svd_dkogbet with the persistent
 *   form and flags = 0, except that the block size is the one already tuned by an earlier
 *   k2svd_dkogbet call on the device, or a default (results do not depend on it).
 *   A problem whose scratch would exceed the array is rejected with K2SVD_ENOSPACE before
 *   anything is launched; the scratch is 32 * batch bytes plus 8 * (n^2 + 1) bytes for
 *   each order n above 128, each part rounded up to 256 bytes, plus 512 bytes (so up to
 *   32752 matrices of orders <= 128).
 *   The first call on a device looks up the address of that device's array with the device
 *   current.  The call uploads its descriptor table from a static host array with a
 *   cudaMemcpyAsync from pageable memory, which CUDA performs synchronously with respect to
 *   the host: the call returns only after the work already queued on `stream` has finished.
 *   The call cannot be captured into a CUDA graph (K2SVD_ECAPTURE).
 *   All calls share the array and each call overwrites it: calls whose work overlaps on a
 *   GPU (other streams, other host threads) race.  Serialize them, e.g. on one stream.
 */
#define K2SVD_ENOSPACE (-1001)
#define K2SVD_KOG_NOALLOC_BYTES (1 << 20)
int k2svd_dkogbet_noalloc(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs,
                          const double *A, double *U, double *V, double *S, int32_t *sweeps, int32_t *info,
                          int32_t max_sweeps, double tol_factor, void *stream);

/*
 * k2svd_dkog_sigma_bwd / k2svd_skog_sigma_bwd -- gradient of the singular values of the
 * k2svd_?kogbet batch with respect to A: dA_i = U_i diag(dS_i) V_i^T (sigma = diag(U^T A V)
 * with U, V held fixed; no paper counterpart).  Same n/offs/soffs description as
 * k2svd_?kogbet; dS holds n[i] values per matrix at soffs[i]; dA is written like A.
 * Element (r, c) is the sum over q = 0..n-1 in increasing order of (U_rq dS_q) V_cq with
 * fma (bitwise reproducible).  batch <= 65535.  workspace: device scratch of at least
 * 32 * batch bytes, 256-byte aligned (the k2svd_?kogbet workspace is large enough).
 * Argument order for error codes: 1 batch, 2 n, 3 offs, 4 soffs, 5 U, 6 V, 7 dS, 8 dA,
 * 9 workspace, 10 ws_bytes.  K2SVD_ECAPTURE on a stream that is being captured.
 */
int k2svd_dkog_sigma_bwd(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs,
                         const double *U, const double *V, const double *dS, double *dA,
                         void *workspace, size_t ws_bytes, void *stream);
int k2svd_skog_sigma_bwd(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs,
                         const float *U, const float *V, const float *dS, float *dA,
                         void *workspace, size_t ws_bytes, void *stream);

/*
 * k2svd_version -- library version as major*10000 + minor*100 + patch.
 */
int k2svd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* K2SVD_H */
