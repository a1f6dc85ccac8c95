// Backward (adjoint) of the batched 2x2 SVD: k2svd_{d,s}gesvd2_bwd (include/k2svd.h).
// One matrix per thread, SoA planes, persistent grid; a streaming kernel (reads 20
// elements, writes 4 per matrix).
#include <cstdint>
#include <cuda_runtime.h>

#include "k2_fp.cuh"
#include "k2svd.h"
#include "k2_launch.h"

namespace k2 {

template <typename T> struct bwd_args {
    const T *u0, *u1, *u2, *u3, *s1, *s2, *v0, *v1, *v2, *v3;
    const T *ds1, *ds2, *du0, *du1, *du2, *du3, *dv0, *dv1, *dv2, *dv3;
    T *g0, *g1, *g2, *g3;
    T tau;
    int64_t n;
};

template <typename T>
__global__ void __launch_bounds__(256) bwd_kernel(const bwd_args<T> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const T u11 = a.u0[i], u21 = a.u1[i], u12 = a.u2[i], u22 = a.u3[i];
        const T v11 = a.v0[i], v21 = a.v1[i], v12 = a.v2[i], v22 = a.v3[i];
        const T s1 = a.s1[i], s2 = a.s2[i];
        const T d1 = a.ds1 ? a.ds1[i] : T(0), d2 = a.ds2 ? a.ds2[i] : T(0);
        T am = T(0), bm = T(0);
        if (a.du0) {       // a = (U^T dU)_12 - (U^T dU)_21
            const T e11 = a.du0[i], e21 = a.du1[i], e12 = a.du2[i], e22 = a.du3[i];
            am = fma(u11, e12, u21 * e22) - fma(u12, e11, u22 * e21);
        }
        if (a.dv0) {       // b = (V^T dV)_12 - (V^T dV)_21
            const T e11 = a.dv0[i], e21 = a.dv1[i], e12 = a.dv2[i], e22 = a.dv3[i];
            bm = fma(v11, e12, v21 * e22) - fma(v12, e11, v22 * e21);
        }
        T m12 = T(0), m21 = T(0);
        // comparisons, the maximum and the division run on the integer pipes (the FP64
        // pipe is the scarce one); the results are those of the IEEE operations
        if (!is_fin(s1) || !is_fin(s2)) {
            m12 = m21 = T(NAN);
        } else if (gt0(s1)) {
            // scale by 2^-k with s1 2^-k in [1,2): F12 (a s2 + b s1) = -(a s2' + b s1') / (g' s') 2^-k
            int k; T f;
            fpt<T>::split(s1, k, f);
            const T s1n = f, s2n = fpt<T>::scale(s2, -k);
            const T d = s1n - s2n, t = a.tau * s1n;              // both >= 0
            const T gap = pos_lt(d, t) ? t : d;
            const T q = qdiv(T(1), gap * (s1n + s2n));
            m12 = fpt<T>::scale(-fma(am, s2n, bm * s1n) * q, -k);
            m21 = fpt<T>::scale(-fma(am, s1n, bm * s2n) * q, -k);
        }
        // W = U M, dG = W V^T
        const T w11 = fma(u12, m21, u11 * d1), w21 = fma(u22, m21, u21 * d1);
        const T w12 = fma(u12, d2, u11 * m12), w22 = fma(u22, d2, u21 * m12);
        a.g0[i] = fma(w12, v12, w11 * v11);
        a.g1[i] = fma(w22, v12, w21 * v11);
        a.g2[i] = fma(w12, v22, w11 * v21);
        a.g3[i] = fma(w22, v22, w21 * v21);
    }
}

template <typename T>
static int gesvd2_bwd(int64_t n, const T *U, const T *S, const T *V, int64_t ld, const T *dS, const T *dU,
                      const T *dV, T *dG, T tau, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!U) return -2;
    if (!S) return -3;
    if (!V) return -4;
    if (ld < n) return -5;
    if (!dG) return -9;
    if (!(tau >= T(0))) return -10;
    bwd_args<T> a;
    a.u0 = U; a.u1 = U + ld; a.u2 = U + 2 * ld; a.u3 = U + 3 * ld;
    a.v0 = V; a.v1 = V + ld; a.v2 = V + 2 * ld; a.v3 = V + 3 * ld;
    a.s1 = S; a.s2 = S + ld;
    a.ds1 = dS; a.ds2 = dS ? dS + ld : nullptr;
    a.du0 = dU; a.du1 = dU ? dU + ld : nullptr; a.du2 = dU ? dU + 2 * ld : nullptr; a.du3 = dU ? dU + 3 * ld : nullptr;
    a.dv0 = dV; a.dv1 = dV ? dV + ld : nullptr; a.dv2 = dV ? dV + 2 * ld : nullptr; a.dv3 = dV ? dV + 3 * ld : nullptr;
    a.g0 = dG; a.g1 = dG + ld; a.g2 = dG + 2 * ld; a.g3 = dG + 3 * ld;
    a.tau = tau; a.n = n;
    static thread_local int cached_dev = -1, cached_blocks = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cached_dev) {
        int nb = 0;
        if (grid_for(bwd_kernel<T>, 256, 0, &nb) != 0) return K2SVD_ECUDA;
        cached_dev = dev; cached_blocks = nb;
    }
    int64_t need = (n + 255) / 256;
    int blocks = (int)(need < cached_blocks ? need : cached_blocks);
    bwd_kernel<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

}  // namespace k2

extern "C" {

int k2svd_dgesvd2_bwd(int64_t batch, const double *U, const double *S, const double *V, int64_t ld,
                      const double *dS, const double *dU, const double *dV, double *dG, double gap_rtol, void *stream)
{
    return k2::gesvd2_bwd<double>(batch, U, S, V, ld, dS, dU, dV, dG, gap_rtol, stream);
}

int k2svd_sgesvd2_bwd(int64_t batch, const float *U, const float *S, const float *V, int64_t ld,
                      const float *dS, const float *dU, const float *dV, float *dG, float gap_rtol, void *stream)
{
    return k2::gesvd2_bwd<float>(batch, U, S, V, ld, dS, dU, dV, dG, gap_rtol, stream);
}

}  // extern "C"
