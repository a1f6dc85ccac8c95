// The SVD of rectangular matrices (Sect. 1): k2svd_{d,s}gesvdr and k2svd_{d,s}gesvdr_ws,
// declared in include/k2svd.h.  An m x n matrix is reduced to a square one by Householder
// QR with column pivoting (for m < n, of its transpose), the batched n x n Kogbetliantz
// driver (k2_kog.cu) decomposes the triangular factors, and U, V are assembled.
//
// Every step follows one fixed order of correctly rounded operations, so the results are
// reproducible and equal to the oracle's:
//   * B = A or A^T (p x q, p >= q), scaled by the power of two 2^k that brings its largest
//     element into [1/2, 1);
//   * step j: each thread recomputes the squared norms of its columns over rows j..p-1 (fma
//     in increasing row order); one thread takes the first column of largest norm as the
//     pivot, swaps it in, and forms the reflector: alpha = -sign(x0) ||x||, v0 = x0 - alpha,
//     v^T v = 2 (||x|| (||x|| + |x0|)); each thread then applies it to its columns
//     (s = v0 y0 and fma in row order, f = (s + s) / v^T v, y <- fma(-f, v, y));
//   * Q = H_0 ... H_{q-1} [I; 0] with the same formulas, reflectors in reverse order;
//   * U = Q U_R (fma over k in increasing order), V = P V_R (row j of V_R to row perm[j]);
//     for m < n the two exchange places; sigma = 2^-k sigma_R.
// One block per matrix, its columns spread over the threads; the working matrices live in
// the workspace.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "k2_fp.cuh"
#include "k2svd.h"
#include "k2_launch.h"

namespace k2 {

struct rect_desc {
    int32_t m, n, p, q, tr, idx;
    int64_t aoff, uoff, voff, soff;     // caller's A, U, V, S
    int64_t boff;                       // B and Q (p q elements each) in the workspace
    int64_t roff, sroff;                // R, U_R, V_R (q q each, packed) and sigma_R (q)
    int64_t woff;                       // perm, norms, v^T v, alpha: 4 q words
};

template <typename T> struct rect_params {
    const rect_desc *desc;
    int count;
    const T *A;
    T *U, *V, *S;
    T *B, *Q, *R, *UR, *VR, *SR;
    T *wv;                              // norms, v^T v, alphas (3 q per matrix at woff)
    int32_t *perm;                      // q per matrix at woff
    int32_t *kscale;                    // per matrix
};

// B and the Q being formed are row-major in the workspace (element (r, c) at r q + c): each
// thread owns columns and walks down them in row order, as the fixed operation order asks,
// and at every row the threads of a warp touch consecutive addresses.  Q is then copied
// column-major into B's place for the assembly.
template <typename T>
__global__ void __launch_bounds__(128) qrcp_kernel(const rect_params<T> P)
{
    __shared__ int s_emax, s_piv;
    for (int mi = blockIdx.x; mi < P.count; mi += gridDim.x) {
        const rect_desc d = P.desc[mi];
        const int p = d.p, q = d.q, tid = threadIdx.x, nt = blockDim.x;
        T *B = P.B + d.boff, *Q = P.Q + d.boff;
        T *nrm = P.wv + 3 * d.woff, *vv = nrm + q, *alph = vv + q;
        int32_t *perm = P.perm + d.woff;
        const T *A = P.A + d.aoff;
        if (tid == 0) s_emax = INT_MIN;
        __syncthreads();
        int le = INT_MIN;
        for (int64_t e = tid; e < (int64_t)p * q; e += nt) {
            const int r = (int)(e / q), c = (int)(e % q);
            const T x = d.tr ? A[(int64_t)r * d.m + c] : A[(int64_t)c * d.m + r];
            B[e] = x;
            if (is_fin(x) && !eq0(x)) le = max(le, fpt<T>::expo(x));
        }
        if (le != INT_MIN) atomicMax(&s_emax, le);
        __syncthreads();
        const int k = s_emax == INT_MIN ? 0 : -(s_emax + 1);
        for (int64_t e = tid; e < (int64_t)p * q; e += nt) B[e] = fpt<T>::scale(B[e], k);
        for (int c = tid; c < q; c += nt) perm[c] = c;
        if (tid == 0) P.kscale[mi] = k;
        __syncthreads();
        for (int j = 0; j < q; ++j) {
            for (int c = j + tid; c < q; c += nt) {
                T sq = T(0);
                for (int r = j; r < p; ++r) { const T b = B[(int64_t)r * q + c]; sq = fma(b, b, sq); }
                nrm[c] = sq;
            }
            __syncthreads();
            if (tid == 0) {
                int piv = j;
                for (int c = j + 1; c < q; ++c) if (nrm[c] > nrm[piv]) piv = c;
                s_piv = piv;
            }
            __syncthreads();
            const int piv = s_piv;
            if (piv != j) {
                for (int r = tid; r < p; r += nt) {
                    T *row = B + (int64_t)r * q;
                    const T t = row[j]; row[j] = row[piv]; row[piv] = t;
                }
                if (tid == 0) { const int t = perm[j]; perm[j] = perm[piv]; perm[piv] = t; }
            }
            __syncthreads();
            T *x = B + (int64_t)j * q + j;                     // x[i q] = element (j + i, j)
            const int L = p - j;
            if (tid == 0) {
                if (nrm[piv] == T(0)) { vv[j] = T(0); alph[j] = x[0]; }
                else {
                    const T nx = sqrt(nrm[piv]);
                    const T x0 = x[0];
                    const T alpha = (x0 < T(0)) ? nx : -nx;
                    alph[j] = alpha;
                    vv[j] = T(2) * (nx * (nx + fabs(x0)));
                    x[0] = x0 - alpha;
                }
            }
            __syncthreads();
            const T w = vv[j];
            if (w != T(0)) {
                for (int c = j + 1 + tid; c < q; c += nt) {
                    T *y = B + (int64_t)j * q + c;                 // y[i q] = element (j + i, c)
                    T s = x[0] * y[0];
                    for (int i = 1; i < L; ++i) s = fma(x[(int64_t)i * q], y[(int64_t)i * q], s);
                    const T f = (s + s) / w;
                    for (int i = 0; i < L; ++i) y[(int64_t)i * q] = fma(-f, x[(int64_t)i * q], y[(int64_t)i * q]);
                }
            }
            __syncthreads();
        }
        // R (q x q column-major, packed for the n x n driver) and Q = H_0 ... H_{q-1} [I; 0]
        T *R = P.R + d.roff;
        for (int64_t e = tid; e < (int64_t)q * q; e += nt) {
            const int c = (int)(e / q), r = (int)(e % q);
            R[e] = r < c ? B[(int64_t)r * q + c] : (r == c ? alph[c] : T(0));
        }
        for (int64_t e = tid; e < (int64_t)p * q; e += nt) {
            const int r = (int)(e / q), c = (int)(e % q);
            Q[e] = r == c ? T(1) : T(0);
        }
        __syncthreads();
        for (int j = q - 1; j >= 0; --j) {
            const T w = vv[j];
            if (w == T(0)) continue;
            const T *x = B + (int64_t)j * q + j;
            const int L = p - j;
            for (int c = tid; c < q; c += nt) {
                T *y = Q + (int64_t)j * q + c;
                T s = x[0] * y[0];
                for (int i = 1; i < L; ++i) s = fma(x[(int64_t)i * q], y[(int64_t)i * q], s);
                const T f = (s + s) / w;
                for (int i = 0; i < L; ++i) y[(int64_t)i * q] = fma(-f, x[(int64_t)i * q], y[(int64_t)i * q]);
            }
            __syncthreads();
        }
        // Q column-major into B's place (the reflectors are no longer needed)
        for (int64_t e = tid; e < (int64_t)p * q; e += nt) {
            const int c = (int)(e / p), r = (int)(e % p);
            B[e] = Q[(int64_t)r * q + c];
        }
        __syncthreads();
    }
}

// U = Q U_R and V = P V_R (exchanged for m < n); sigma = 2^-k sigma_R
template <typename T>
__global__ void __launch_bounds__(256) rect_assemble_kernel(const rect_params<T> P)
{
    for (int mi = blockIdx.x; mi < P.count; mi += gridDim.x) {
        const rect_desc d = P.desc[mi];
        const int p = d.p, q = d.q, tid = threadIdx.x, nt = blockDim.x;
        const T *Q = P.B + d.boff;                        // column-major Q, left there by qrcp_kernel
        const T *UR = P.UR + d.roff, *VR = P.VR + d.roff, *SR = P.SR + d.sroff;
        const int32_t *perm = P.perm + d.woff;
        T *QU = d.tr ? P.V + d.voff : P.U + d.uoff;
        T *PV = d.tr ? P.U + d.uoff : P.V + d.voff;
        for (int64_t e = tid; e < (int64_t)p * q; e += nt) {
            const int c = (int)(e / p), r = (int)(e % p);
            const T *u = UR + (int64_t)c * q;
            T acc = Q[r] * u[0];
            for (int t = 1; t < q; ++t) acc = fma(Q[(int64_t)t * p + r], u[t], acc);
            QU[e] = acc;
        }
        for (int64_t e = tid; e < (int64_t)q * q; e += nt) {
            const int c = (int)(e / q), j = (int)(e % q);
            PV[(int64_t)c * q + perm[j]] = VR[e];
        }
        const int k = P.kscale[mi];
        for (int c = tid; c < q; c += nt) P.S[d.soff + c] = is_fin(SR[c]) ? fpt<T>::scale(SR[c], -k) : SR[c];
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T> struct rect_plan {
    std::vector<rect_desc> desc;
    std::vector<int32_t> qs;
    std::vector<int64_t> roffs, sroffs;
    size_t off_desc, off_B, off_Q, off_R, off_UR, off_VR, off_SR, off_wv, off_perm, off_k, off_kog, kog_bytes, total;
};

template <typename T>
static int rect_make_plan(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, rect_plan<T> &pl)
{
    pl.desc.resize((size_t)batch);
    pl.qs.resize((size_t)batch);
    pl.roffs.resize((size_t)batch);
    pl.sroffs.resize((size_t)batch);
    int64_t b = 0, r = 0, sr = 0, w = 0;
    for (int64_t i = 0; i < batch; ++i) {
        if (m[i] < 1 || n[i] < 1 || m[i] > 65536 || n[i] > 65536) return -2;
        rect_desc &d = pl.desc[(size_t)i];
        d.m = m[i]; d.n = n[i]; d.tr = m[i] < n[i] ? 1 : 0;
        d.p = d.tr ? n[i] : m[i]; d.q = d.tr ? m[i] : n[i];
        if (d.q > 4096) return -2;
        d.idx = (int32_t)i;
        d.boff = b; b += ((int64_t)d.p * d.q + 1) & ~(int64_t)1;
        d.roff = r; r += (int64_t)d.q * d.q;
        d.sroff = sr; sr += d.q;
        d.woff = w; w += d.q;
        pl.qs[(size_t)i] = d.q; pl.roffs[(size_t)i] = d.roff; pl.sroffs[(size_t)i] = d.sroff;
    }
    size_t kb = 0;
    const int rc = sizeof(T) == 8 ? k2svd_dkogbet_ws(batch, pl.qs.data(), flags, &kb)
                                  : k2svd_skogbet_ws(batch, pl.qs.data(), flags, &kb);
    if (rc != 0) return rc;
    size_t off = 0;
    pl.off_desc = off; off = align256(off + (size_t)batch * sizeof(rect_desc));
    pl.off_B = off; off = align256(off + (size_t)b * sizeof(T));
    pl.off_Q = off; off = align256(off + (size_t)b * sizeof(T));
    pl.off_R = off; off = align256(off + (size_t)r * sizeof(T));
    pl.off_UR = off; off = align256(off + (size_t)r * sizeof(T));
    pl.off_VR = off; off = align256(off + (size_t)r * sizeof(T));
    pl.off_SR = off; off = align256(off + (size_t)sr * sizeof(T));
    pl.off_wv = off; off = align256(off + (size_t)3 * w * sizeof(T));
    pl.off_perm = off; off = align256(off + (size_t)w * sizeof(int32_t));
    pl.off_k = off; off = align256(off + (size_t)batch * sizeof(int32_t));
    pl.off_kog = off; pl.kog_bytes = kb; off = align256(off + kb);
    pl.total = off;
    return 0;
}

template <typename T>
static int gesvdr_ws(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    if (batch < 0) return -1;
    if (!ws_bytes) return -5;
    if (batch == 0) { *ws_bytes = 0; return 0; }
    if (!m) return -2;
    if (!n) return -3;
    rect_plan<T> pl;
    const int rc = rect_make_plan<T>(batch, m, n, flags, pl);
    if (rc != 0) return rc == -2 ? -2 : rc;
    *ws_bytes = pl.total;
    return 0;
}

template <typename T>
static int gesvdr(int64_t batch, const int32_t *m, const int32_t *n, const int64_t *aoffs, const int64_t *uoffs,
                  const int64_t *voffs, const int64_t *soffs, const T *A, T *U, T *V, T *S, int32_t *sweeps,
                  int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags, void *workspace,
                  size_t ws_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (batch == 0) return 0;
    if (!m) return -2;
    if (!n) return -3;
    if (!aoffs) return -4;
    if (!uoffs) return -5;
    if (!voffs) return -6;
    if (!soffs) return -7;
    if (!A) return -8;
    if (!U) return -9;
    if (!V) return -10;
    if (!S) return -11;
    if (max_sweeps < 0) return -14;
    if (!(tol_factor > 0)) return -15;
    if (flags & ~(K2SVD_KOG_NOTUNE)) return -16;
    if (!workspace || ((uintptr_t)workspace & 255)) return -17;
    rect_plan<T> pl;
    int rc = rect_make_plan<T>(batch, m, n, flags, pl);
    if (rc != 0) return rc;
    if (ws_bytes < pl.total) return -18;
    for (int64_t i = 0; i < batch; ++i) {
        rect_desc &d = pl.desc[(size_t)i];
        d.aoff = aoffs[i]; d.uoff = uoffs[i]; d.voff = voffs[i]; d.soff = soffs[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = capture_guard(st)) != 0) return rc;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    if (cudaMemcpyAsync(ws + pl.off_desc, pl.desc.data(), pl.desc.size() * sizeof(rect_desc), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return K2SVD_ECUDA;
    rect_params<T> P;
    P.desc = reinterpret_cast<const rect_desc *>(ws + pl.off_desc);
    P.count = (int)batch;
    P.A = A; P.U = U; P.V = V; P.S = S;
    P.B = reinterpret_cast<T *>(ws + pl.off_B);
    P.Q = reinterpret_cast<T *>(ws + pl.off_Q);
    P.R = reinterpret_cast<T *>(ws + pl.off_R);
    P.UR = reinterpret_cast<T *>(ws + pl.off_UR);
    P.VR = reinterpret_cast<T *>(ws + pl.off_VR);
    P.SR = reinterpret_cast<T *>(ws + pl.off_SR);
    P.wv = reinterpret_cast<T *>(ws + pl.off_wv);
    P.perm = reinterpret_cast<int32_t *>(ws + pl.off_perm);
    P.kscale = reinterpret_cast<int32_t *>(ws + pl.off_k);
    int nb = 0;
    if (grid_for(qrcp_kernel<T>, 128, 0, &nb) != 0) return K2SVD_ECUDA;
    qrcp_kernel<T><<<(int)std::min<int64_t>(batch, nb), 128, 0, st>>>(P);
    if (cudaPeekAtLastError() != cudaSuccess) return K2SVD_ECUDA;
    rc = sizeof(T) == 8
        ? k2svd_dkogbet(batch, pl.qs.data(), pl.roffs.data(), pl.sroffs.data(), (const double *)P.R, (double *)P.UR,
                        (double *)P.VR, (double *)P.SR, sweeps, info, max_sweeps, tol_factor, flags,
                        ws + pl.off_kog, pl.kog_bytes, stream)
        : k2svd_skogbet(batch, pl.qs.data(), pl.roffs.data(), pl.sroffs.data(), (const float *)P.R, (float *)P.UR,
                        (float *)P.VR, (float *)P.SR, sweeps, info, max_sweeps, tol_factor, flags,
                        ws + pl.off_kog, pl.kog_bytes, stream);
    if (rc != 0) return rc == K2SVD_ECUDA ? K2SVD_ECUDA : -19;   // rejected by the square driver
    if (grid_for(rect_assemble_kernel<T>, 256, 0, &nb) != 0) return K2SVD_ECUDA;
    rect_assemble_kernel<T><<<(int)std::min<int64_t>(batch, nb), 256, 0, st>>>(P);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

}  // namespace k2

extern "C" {

int k2svd_dgesvdr_ws(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    return k2::gesvdr_ws<double>(batch, m, n, flags, ws_bytes);
}

int k2svd_sgesvdr_ws(int64_t batch, const int32_t *m, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    return k2::gesvdr_ws<float>(batch, m, n, flags, ws_bytes);
}

int k2svd_dgesvdr(int64_t batch, const int32_t *m, const int32_t *n, const int64_t *aoffs, const int64_t *uoffs,
                  const int64_t *voffs, const int64_t *soffs, const double *A, double *U, double *V, double *S,
                  int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream)
{
    return k2::gesvdr<double>(batch, m, n, aoffs, uoffs, voffs, soffs, A, U, V, S, sweeps, info, max_sweeps,
                              tol_factor, flags, workspace, ws_bytes, stream);
}

int k2svd_sgesvdr(int64_t batch, const int32_t *m, const int32_t *n, const int64_t *aoffs, const int64_t *uoffs,
                  const int64_t *voffs, const int64_t *soffs, const float *A, float *U, float *V, float *S,
                  int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream)
{
    return k2::gesvdr<float>(batch, m, n, aoffs, uoffs, voffs, soffs, A, U, V, S, sweeps, info, max_sweeps,
                             tol_factor, flags, workspace, ws_bytes, stream);
}

}  // extern "C"
