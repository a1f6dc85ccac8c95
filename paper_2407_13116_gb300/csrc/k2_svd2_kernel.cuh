// The batched 2x2 SVD kernel (arXiv 2407.13116, Sect. 3) and its host-side argument checks,
// shared by the translation units of the correctly rounded method (k2_gesvd2.cu) and of the
// variant with the hypot that is not correctly rounded (k2_ncr.cu).
//
// One matrix per thread.  Inputs and outputs are SoA planes, so every load and store of a
// warp touches 32 consecutive elements of one plane (fully coalesced).  The grid is
// persistent: (SM count) x (resident blocks per SM) blocks stride over the batch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "k2_svd2.cuh"
#include "k2svd.h"
#include "k2_launch.h"

namespace k2 {

template <typename T> struct svd_args {
    const T *g0, *g1, *g2, *g3;       // g11 g21 g12 g22 (trsvd2: F, -, Gu, H)
    T *u0, *u1, *u2, *u3, *v0, *v1, *v2, *v3;
    T *s1, *s2;
    int32_t *se1, *se2;
    T *sf1, *sf2;
    int32_t *info;
    int64_t n;
};

template <typename T> __device__ __forceinline__ T pz(T x) { return unneg0(x); }   // -0 -> +0

// Blocks of 256 threads with at most 32 registers a thread, so 8 blocks (64 warps, the full
// occupancy) are resident per SM.  The rest of the FP64 state spills to local memory (L1):
// on a GB300 this is 7% faster than 64 registers at half occupancy (which was 5% faster than
// the unconstrained 80-register build), as the extra warps hide the instruction-fetch
// stalls of the divergent method.  One exception, also measured: the triangular FP64 kernel
// of the variant with the hypot that is not correctly rounded runs 2.8 times slower at 32
// registers than at 64, so it keeps blocks of 128 threads (8 per SM, 64 registers).
template <typename T, bool TRI, bool NCR> constexpr int svd2_threads()
{
    return (sizeof(T) == 8 && TRI && NCR) ? 128 : 256;
}
// NCR: the method with the hypot that is not correctly rounded (Alg. 1's branch for it).
// Inputs and outputs are touched once: streaming loads and stores (__ldcs, __stcs) keep them
// from evicting the spilled registers from L2, which cut the kernel's DRAM traffic by a
// quarter (reads down to the input bytes) at the same speed.
template <typename T, bool TRI, bool NCR>
__global__ void __launch_bounds__(svd2_threads<T, TRI, NCR>(), 8) svd2_kernel(const svd_args<T> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const T g11 = __ldcs(a.g0 + i);
        const T g21 = TRI ? T(0) : __ldcs(a.g1 + i);
        const T g12 = __ldcs(a.g2 + i);
        const T g22 = __ldcs(a.g3 + i);
        svd2_out<T> o;
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22)) {
            svd2<T, !TRI, NCR>(g11, g21, g12, g22, o);         // general matrices leave the FP64 pipe room
        } else {
            const T qn = T(NAN);
            o.U.a11 = o.U.a21 = o.U.a12 = o.U.a22 = qn;
            o.V.a11 = o.V.a21 = o.V.a12 = o.V.a22 = qn;
            o.s1.e = o.s2.e = 0; o.s1.f = o.s2.f = qn;
            o.info = -1;
        }
        __stcs(a.u0 + i, pz(o.U.a11)); __stcs(a.u1 + i, pz(o.U.a21)); __stcs(a.u2 + i, pz(o.U.a12)); __stcs(a.u3 + i, pz(o.U.a22));
        __stcs(a.v0 + i, pz(o.V.a11)); __stcs(a.v1 + i, pz(o.V.a21)); __stcs(a.v2 + i, pz(o.V.a12)); __stcs(a.v3 + i, pz(o.V.a22));
        if (o.info >= 0) {
            __stcs(a.s1 + i, ef_fl(o.s1)); __stcs(a.s2 + i, ef_fl(o.s2));
        } else {
            __stcs(a.s1 + i, o.s1.f); __stcs(a.s2 + i, o.s2.f);
        }
        if (a.se1) { __stcs(a.se1 + i, o.s1.e); __stcs(a.se2 + i, o.s2.e); }
        if (a.sf1) { __stcs(a.sf1 + i, o.s1.f); __stcs(a.sf2 + i, o.s2.f); }
        if (a.info) __stcs(a.info + i, o.info);
    }
}

template <typename T, bool TRI, bool NCR>
static int launch(const svd_args<T> &a, cudaStream_t st)
{
    static thread_local int cached_dev = -1, cached_blocks = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cached_dev) {
        int nb = 0;
        if (grid_for(svd2_kernel<T, TRI, NCR>, svd2_threads<T, TRI, NCR>(), 0, &nb) != 0) return K2SVD_ECUDA;
        cached_dev = dev; cached_blocks = nb;
    }
    constexpr int nt = svd2_threads<T, TRI, NCR>();
    int64_t need = (a.n + nt - 1) / nt;
    int blocks = (int)(need < cached_blocks ? need : cached_blocks);
    svd2_kernel<T, TRI, NCR><<<blocks, nt, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

template <typename T, bool NCR>
static int gesvd2(int64_t n, const T *G, int64_t ldg, T *U, int64_t ldu, T *V, int64_t ldv,
                  T *S, int64_t lds, int32_t *Se, T *Sf, int32_t *info, void *stream)
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
    svd_args<T> a;
    a.g0 = G; a.g1 = G + ldg; a.g2 = G + 2 * ldg; a.g3 = G + 3 * ldg;
    a.u0 = U; a.u1 = U + ldu; a.u2 = U + 2 * ldu; a.u3 = U + 3 * ldu;
    a.v0 = V; a.v1 = V + ldv; a.v2 = V + 2 * ldv; a.v3 = V + 3 * ldv;
    a.s1 = S; a.s2 = S + lds;
    a.se1 = Se; a.se2 = Se ? Se + lds : nullptr;
    a.sf1 = Sf; a.sf2 = Sf ? Sf + lds : nullptr;
    a.info = info; a.n = n;
    return launch<T, false, NCR>(a, (cudaStream_t)stream);
}

template <typename T, bool NCR>
static int trsvd2(int64_t n, const T *F, const T *Gu, const T *H, T *U, int64_t ldu, T *V, int64_t ldv,
                  T *S, int64_t lds, int32_t *Se, T *Sf, int32_t *info, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!F) return -2;
    if (!Gu) return -3;
    if (!H) return -4;
    if (!U) return -5;
    if (ldu < n) return -6;
    if (!V) return -7;
    if (ldv < n) return -8;
    if (!S) return -9;
    if (lds < n) return -10;
    svd_args<T> a;
    a.g0 = F; a.g1 = nullptr; a.g2 = Gu; a.g3 = H;
    a.u0 = U; a.u1 = U + ldu; a.u2 = U + 2 * ldu; a.u3 = U + 3 * ldu;
    a.v0 = V; a.v1 = V + ldv; a.v2 = V + 2 * ldv; a.v3 = V + 3 * ldv;
    a.s1 = S; a.s2 = S + lds;
    a.se1 = Se; a.se2 = Se ? Se + lds : nullptr;
    a.sf1 = Sf; a.sf2 = Sf ? Sf + lds : nullptr;
    a.info = info; a.n = n;
    return launch<T, true, NCR>(a, (cudaStream_t)stream);
}

}  // namespace k2
