// The SVD of complex 2x2 matrices (arXiv 2407.13116, Sect. 3.4): k2svd_zgesvd2 (double) and
// k2svd_cgesvd2 (float), declared in include/k2svd.h.
//
// Real input takes the real method; purely imaginary input G = iH the real method on H with
// U = i U_H.  Otherwise the matrix is made real by unitary transformations and the real
// method (svd2 of k2_svd2.cuh) runs on the result:
//   * phase 1 over every real and imaginary component with the scale type raised by one
//     (Sect. 3.4 item 1);
//   * at most three nonzeros: row and column phases conj(z)/|z| make every element real and
//     positive (each phase fixed once, in the order of the real method's sign extraction);
//   * no zeros: complex column norms and column pivoting, row phases for a real first
//     column, row pivoting, the real rotation of eq. (QR15) without (EXT) (item 3), then a
//     column phase for r12 and a row phase for r22;
//   * U and V assembled from the phases, the permutations, the rotation and the real
//     singular vectors by real-complex products (item 2).
// Every step is one correctly rounded real operation in a fixed order, so the result is
// bitwise reproducible: complex product (a,b)(c,d) = (fma(a, c, -(b d)), fma(a, d, b c)),
// |z| = the correctly rounded hypot, conj(z)/|z| as two quotients.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "k2_svd2.cuh"
#include "k2svd.h"
#include "k2_launch.h"

namespace k2 {

template <typename T> struct cx { T re, im; };

template <typename T> __device__ __forceinline__ cx<T> mkc(T re, T im) { cx<T> z; z.re = re; z.im = im; return z; }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return mkc(fma(a.re, b.re, ngt(a.im * b.im)), fma(a.re, b.im, a.im * b.re));
}
template <typename T> __device__ __forceinline__ bool cnz(cx<T> z) { return !eq0(z.re) || !eq0(z.im); }
template <typename T> __device__ __forceinline__ T cabs(cx<T> z) { return hypot_cr(z.re, z.im); }
// conj(z)/|z| for z != 0
template <typename T> __device__ __forceinline__ cx<T> cphase(cx<T> z, T az) { return mkc(qdiv(z.re, az), qdiv(ngt(z.im), az)); }
template <typename T> __device__ __forceinline__ cx<T> cconj(cx<T> z) { return mkc(z.re, ngt(z.im)); }

template <typename T> struct cm22 { cx<T> a11, a21, a12, a22; };

template <typename T> __device__ __forceinline__ cm22<T> cm_of(const m22<T> &m)
{
    cm22<T> c;
    c.a11 = mkc(m.a11, T(0)); c.a21 = mkc(m.a21, T(0)); c.a12 = mkc(m.a12, T(0)); c.a22 = mkc(m.a22, T(0));
    return c;
}
// diag(d0, d1) A
template <typename T> __device__ __forceinline__ void cm_rows(cm22<T> &A, cx<T> d0, cx<T> d1)
{
    A.a11 = cmul(d0, A.a11); A.a12 = cmul(d0, A.a12);
    A.a21 = cmul(d1, A.a21); A.a22 = cmul(d1, A.a22);
}
// element (i, j) of M B, M complex, B real: fma(M[i][1], B[1][j], M[i][0] B[0][j]) per part
template <typename T> __device__ __forceinline__ cx<T> cm_dot(cx<T> m0, cx<T> m1, T b0, T b1)
{
    return mkc(fma(m1.re, b1, m0.re * b0), fma(m1.im, b1, m0.im * b0));
}
template <typename T> __device__ __forceinline__ void cm_swap_rows(cm22<T> &A)
{
    cx<T> t = A.a11; A.a11 = A.a21; A.a21 = t;
    t = A.a12; A.a12 = A.a22; A.a22 = t;
}

template <typename T> struct cres {
    cm22<T> U, V;
    ef<T> s1, s2;
    int info;
};

constexpr int CF_IMAG = 0x100;   // purely imaginary G
constexpr int CF_CPLX = 0x200;   // the complex reduction

template <typename T>
__device__ __forceinline__ int cpattern(const cx<T> g[4])    // g11, g21, g12, g22
{
    return cnz(g[0]) | (cnz(g[1]) << 1) | (cnz(g[2]) << 2) | (cnz(g[3]) << 3);
}

// The complex reduction; g (g11, g21, g12, g22) has a nonzero real and a nonzero imaginary part.
template <typename T>
__device__ void csvd2(cx<T> g[4], cres<T> &o)
{
    const int t = cpattern(g);
    const int cls = cls_of(t);
    int s = 0;
    if (cls != 9) {
        int eG = INT_MIN;
        for (int k = 0; k < 4; ++k) {
            if (!eq0(g[k].re)) eG = max(eG, fpt<T>::expo(g[k].re));
            if (!eq0(g[k].im)) eG = max(eG, fpt<T>::expo(g[k].im));
        }
        s = fpt<T>::ENU - eG - (cls == 15 ? 2 : 1) - 1;
        for (int k = 0; k < 4; ++k) { g[k].re = fpt<T>::scale(g[k].re, s); g[k].im = fpt<T>::scale(g[k].im, s); }
    }
    const int tp = cpattern(g);
    const int clsp = cls_of(tp);
    const cx<T> one = mkc(T(1), T(0));
    cx<T> lam0 = one, lam1 = one, mu0 = one, mu1 = one, l0 = one, l1 = one, lr = one;
    T h11 = T(0), h21 = T(0), h12 = T(0), h22 = T(0);
    bool urv = false, pu = false, pv = false;
    T c = T(1), sn = T(0);
    if (clsp != 15) {
        // w[k] at (row, col) = (k & 1, k >> 1)
        cx<T> w[4] = { g[0], g[1], g[2], g[3] };
        int order[4], no = 0;
        if (clsp == 13) {
            // the upper-triangular arrangement of Sect. 3.2.1: corner a, off-diagonal b (same
            // row as a), opposite corner d (same column as b)
            switch (tp) {
            case 7: order[0] = 2; order[1] = 0; order[2] = 1; break;   // a = g12, b = g11, d = g21
            case 11: order[0] = 3; order[1] = 1; order[2] = 0; break;  // a = g22, b = g21, d = g11
            case 14: order[0] = 1; order[1] = 3; order[2] = 2; break;  // a = g21, b = g22, d = g12
            default: order[0] = 0; order[1] = 2; order[2] = 3; break;  // a = g11, b = g12, d = g22
            }
            no = 3;
        } else {
            // row by row: (0,0), (0,1), (1,0), (1,1)
            const int rowwise[4] = { 0, 2, 1, 3 };
            for (int q = 0; q < 4; ++q)
                if (cnz(w[rowwise[q]])) order[no++] = rowwise[q];
        }
        bool rowset0 = false, rowset1 = false;
        for (int q = 0; q < no; ++q) {
            const int k = order[q], i = k & 1, j = k >> 1;
            const cx<T> z = w[k];
            const T az = cabs(z);
            const cx<T> rho = cphase(z, az);
            const bool rowfree = i ? !rowset1 : !rowset0;
            if (rowfree) {
                if (i) { rowset1 = true; lam1 = rho; } else { rowset0 = true; lam0 = rho; }
                const int other = i | ((1 - j) << 1);              // (i, 1-j)
                w[other] = cmul(w[other], rho);
            } else {
                if (j) mu1 = rho; else mu0 = rho;
                const int other = (1 - i) | (j << 1);              // (1-i, j)
                w[other] = cmul(w[other], rho);
            }
            w[k] = mkc(az, T(0));
        }
        h11 = w[0].re; h21 = w[1].re; h12 = w[2].re; h22 = w[3].re;
    } else {
        const T a11 = cabs(g[0]), a21 = cabs(g[1]), a12 = cabs(g[2]), a22 = cabs(g[3]);
        T w1 = hypot_cr(a11, a21), w2 = hypot_cr(a12, a22);
        cx<T> x11 = g[0], x21 = g[1], x12 = g[2], x22 = g[3];
        T b1 = a11, b2 = a21;
        if (pos_lt(w1, w2)) {
            pv = true;
            cx<T> t0 = x11; x11 = x12; x12 = t0;
            t0 = x21; x21 = x22; x22 = t0;
            w1 = w2;
            b1 = a12; b2 = a22;
        }
        l0 = cphase(x11, b1);
        l1 = cphase(x21, b2);
        cx<T> y12 = cmul(x12, l0), y22 = cmul(x22, l1);
        T y11 = b1, y21 = b2;
        if (pos_lt(y11, y21)) {
            pu = true;
            T tt = y11; y11 = y21; y21 = tt;
            cx<T> tz = y12; y12 = y22; y22 = tz;
        }
        const T tth = qdiv(y21, y11);
        const T secth = hypot_cr(tth, T(1));
        c = qdiv(T(1), secth);
        sn = qdiv(tth, secth);
        cx<T> r12 = mkc(qdiv(fma(tth, y22.re, y12.re), secth), qdiv(fma(tth, y22.im, y12.im), secth));
        cx<T> r22 = mkc(qdiv(fma(ngt(tth), y12.re, y22.re), secth), qdiv(fma(ngt(tth), y12.im, y22.im), secth));
        T ar12 = T(0), ar22 = T(0);
        if (cnz(r12)) {
            ar12 = cabs(r12);
            mu1 = cphase(r12, ar12);
            r22 = cmul(r22, mu1);
        }
        if (cnz(r22)) {
            ar22 = cabs(r22);
            lr = cphase(r22, ar22);
        }
        h11 = w1; h12 = ar12; h21 = T(0); h22 = ar22;
        urv = true;
    }
    svd2_out<T> ro;
    svd2<T>(h11, h21, h12, h22, ro);
    o.info = t | (tp << 4) | (((ro.info >> 8) | CF_CPLX) << 8);
    o.s1 = ef_pow2(-s, ro.s1);
    o.s2 = ef_pow2(-s, ro.s2);
    if (!urv) {
        o.U = cm_of(ro.U);
        cm_rows(o.U, cconj(lam0), cconj(lam1));
        o.V = cm_of(ro.V);
        cm_rows(o.V, mu0, mu1);
    } else {
        // U = diag(conj l0, conj l1) P_U U_theta diag(1, conj lr) Uh, U_theta = [[c, -s], [s, c]]
        const cx<T> cl = cconj(lr);
        const cx<T> m00 = mkc(c, T(0)), m10 = mkc(sn, T(0));
        const cx<T> m01 = mkc(ngt(sn) * cl.re, ngt(sn) * cl.im), m11 = mkc(c * cl.re, c * cl.im);
        cm22<T> U;
        U.a11 = cm_dot(m00, m01, ro.U.a11, ro.U.a21);
        U.a12 = cm_dot(m00, m01, ro.U.a12, ro.U.a22);
        U.a21 = cm_dot(m10, m11, ro.U.a11, ro.U.a21);
        U.a22 = cm_dot(m10, m11, ro.U.a12, ro.U.a22);
        if (pu) cm_swap_rows(U);
        cm_rows(U, cconj(l0), cconj(l1));
        o.U = U;
        o.V = cm_of(ro.V);
        cm_rows(o.V, one, mu1);
        if (pv) cm_swap_rows(o.V);
    }
}

template <typename T> struct cargs {
    const T *g;       // 8 planes
    T *u, *v, *s;     // 8, 8, 2 planes
    int32_t *info;
    int64_t ldg, ldu, ldv, lds, n;
};

// Blocks of 256 threads.  double: 8 blocks per SM (full occupancy, 32 registers, the rest of
// the complex reduction spilled to L1-cached local memory) run 25% faster on a GB300 than
// 4 blocks of 128 threads holding everything in 116 registers: the extra warps hide the
// instruction-fetch and latency stalls.  float: 4 blocks of 256 (64 registers).  Streaming
// loads and stores (__ldcs, __stcs), as in svd2_kernel, keep the spills in L2.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 8 : 4) csvd2_kernel(const cargs<T> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        T c8[8];
        bool fin = true, anyim = false, anyre = false;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c8[k] = __ldcs(a.g + k * a.ldg + i);
            fin = fin && is_fin(c8[k]);
            if (!eq0(c8[k])) { if (k & 1) anyim = true; else anyre = true; }
        }
        if (!fin) {
            const T qn = T(NAN);
            for (int k = 0; k < 8; ++k) { __stcs(a.u + k * a.ldu + i, qn); __stcs(a.v + k * a.ldv + i, qn); }
            __stcs(a.s + i, qn); __stcs(a.s + a.lds + i, qn);
            if (a.info) __stcs(a.info + i, -1);
            continue;
        }
        cres<T> o;
        if (!anyim || !anyre) {
            const int k0 = anyim ? 1 : 0;
            svd2_out<T> ro;
            svd2<T>(c8[k0], c8[k0 + 2], c8[k0 + 4], c8[k0 + 6], ro);
            o.U = cm_of(ro.U);
            o.V = cm_of(ro.V);
            if (anyim) {                                       // U = i Uh
                o.U.a11 = mkc(T(0), ro.U.a11); o.U.a21 = mkc(T(0), ro.U.a21);
                o.U.a12 = mkc(T(0), ro.U.a12); o.U.a22 = mkc(T(0), ro.U.a22);
            }
            o.s1 = ro.s1; o.s2 = ro.s2;
            o.info = ro.info | (anyim ? (CF_IMAG << 8) : 0);
        } else {
            cx<T> g[4] = { mkc(c8[0], c8[1]), mkc(c8[2], c8[3]), mkc(c8[4], c8[5]), mkc(c8[6], c8[7]) };
            csvd2(g, o);
        }
        const cx<T> uu[4] = { o.U.a11, o.U.a21, o.U.a12, o.U.a22 }, vv[4] = { o.V.a11, o.V.a21, o.V.a12, o.V.a22 };
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            __stcs(a.u + (2 * e) * a.ldu + i, unneg0(uu[e].re)); __stcs(a.u + (2 * e + 1) * a.ldu + i, unneg0(uu[e].im));
            __stcs(a.v + (2 * e) * a.ldv + i, unneg0(vv[e].re)); __stcs(a.v + (2 * e + 1) * a.ldv + i, unneg0(vv[e].im));
        }
        __stcs(a.s + i, ef_fl(o.s1));
        __stcs(a.s + a.lds + i, ef_fl(o.s2));
        if (a.info) __stcs(a.info + i, o.info);
    }
}

template <typename T>
static int cgesvd2(int64_t n, const T *G, int64_t ldg, T *U, int64_t ldu, T *V, int64_t ldv, T *S, int64_t lds,
                   int32_t *info, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!G) return -2;
    if (ldg < n) return -3;
    if (!U) return -4;
    if (ldu < n) return -5;
    if (!V) return -6;
    if (ldv < n) return -7;
    if (!S) return -8;
    if (lds < n) return -9;
    static thread_local int cdev = -1, cblocks = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cdev) {
        int nb = 0;
        if (grid_for(csvd2_kernel<T>, 256, 0, &nb) != 0) return K2SVD_ECUDA;
        cdev = dev; cblocks = nb;
    }
    cargs<T> a;
    a.g = G; a.u = U; a.v = V; a.s = S; a.info = info;
    a.ldg = ldg; a.ldu = ldu; a.ldv = ldv; a.lds = lds; a.n = n;
    const int64_t need = (n + 255) / 256;
    const int blocks = (int)(need < cblocks ? need : cblocks);
    csvd2_kernel<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

}  // namespace k2

extern "C" {

int k2svd_zgesvd2(int64_t batch, const double *G, int64_t ldg, double *U, int64_t ldu, double *V, int64_t ldv,
                  double *S, int64_t lds, int32_t *info, void *stream)
{
    return k2::cgesvd2<double>(batch, G, ldg, U, ldu, V, ldv, S, lds, info, stream);
}

int k2svd_cgesvd2(int64_t batch, const float *G, int64_t ldg, float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *info, void *stream)
{
    return k2::cgesvd2<float>(batch, G, ldg, U, ldu, V, ldv, S, lds, info, stream);
}

}  // extern "C"
