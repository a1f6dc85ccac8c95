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

// The outputs of matrix i (streaming stores: they are not read again); -0 is stored as +0.
template <typename T> __device__ __forceinline__ void store_out(const svd_args<T> &a, int64_t i, const svd2_out<T> &o)
{
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

// NaN outputs and info = -1 for a matrix with a non-finite element.
template <typename T> __device__ __forceinline__ void nan_out(svd2_out<T> &o)
{
    const T qn = T(NAN);
    o.U.a11 = o.U.a21 = o.U.a12 = o.U.a22 = qn;
    o.V.a11 = o.V.a21 = o.V.a12 = o.V.a22 = qn;
    o.s1.e = o.s2.e = 0; o.s1.f = o.s2.f = qn;
    o.info = -1;
}

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
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22))
            svd2<T, !TRI, NCR>(g11, g21, g12, g22, o);         // general matrices leave the FP64 pipe room
        else
            nan_out(o);
        store_out(a, i, o);
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

// ---------------------------------------------------------------------------------------
// Split form of the FP64 general kernel: phases 1-2 (svd2a_kernel) and phase 3
// (svd2b_kernel) as two launches.  Same operations as the fused kernel, so the same bits.
// Each launch runs part of the method's code, and matrices of classes 13 and 15 meet in one
// copy of Alg. 1 and 2 instead of diverging into two.  Each half also gets its own
// placement of the quotients (SPLIT_FDIV_*).
//
// No scratch memory: the state between the halves (R, tan and sec of theta, s, the
// permutations and signs: svd2_mid, 48 bytes) is parked in the caller's output planes of the
// same matrix -- u11, u21, u12, u22 <- r11, r12, r22, tan theta; v11 <- sec theta;
// sigma1 <- a packed word with the sign bit set -- which phase 3 then overwrites with the
// results.  A final sigma1 is never negative (+0 or above, or a positive NaN for a
// non-finite input), so the sign bit of the sigma1 plane tells phase 3 which matrices are
// still to finish.  Each half runs once over the whole batch.  Measured on a GB300 (2^27
// wide-range matrices): chunks small enough for the parked state to stay in L2 between the
// two launches (3 or 6 rounds of the persistent grid, 45 or 90 MB) took 41.1 and 39.9 ms
// against 38.3 ms for large chunks: each launch's ramp-up and drain cost more than the
// state's DRAM traffic saves (the kernels are bound by their pipes, not by DRAM).
// ---------------------------------------------------------------------------------------
constexpr int64_t SPLIT_MIN = 1 << 16;                    // smaller batches: the fused kernel

// Which quotients use the FP64 divider (csdiv): r12 and r22 of eq. (QR15) in phases 1-2;
// tan theta and every quotient of phase 3 on the integer pipes.  Phases 1-2 are
// integer-heavy (the hypots, eq. (EXT)) and phase 3 FP64-heavy.  Measured on a GB300, 2^27
// wide-range matrices (both halves): 32.8 ms, against 34.8 with tan theta also on the
// divider, 34.0 with only tan theta on it and 33.2 with none (narrow-range 2^26: 22.8, 24.0,
// 22.1, 22.0 ms).
constexpr bool SPLIT_FDIV_A = true, SPLIT_FDIV_AT = false, SPLIT_FDIV_B = false;

// The packed word in the sigma1 plane: bit 63 set (phase 3 pending); bits 0-3 t, 4-7 t',
// 8-15 phase-1-2 flags, 16 c15, 17 pu, 18 pv, 19 na, 20 nb, 21 n12, 22 n22; bits 32-47 the
// prescaling exponent s + 32768 (|s| < 2200).
__device__ __forceinline__ uint64_t mid_pack(const svd2_mid<double> &m)
{
    const uint32_t lo = (uint32_t)(m.t | (m.tp << 4) | (m.flags << 8) | (m.c15 << 16) | (m.pu << 17) | (m.pv << 18) |
                                   (m.na << 19) | (m.nb << 20) | (m.n12 << 21) | (m.n22 << 22));
    return D_SIGN | ((uint64_t)(uint32_t)(m.s + 32768) << 32) | lo;
}
__device__ __forceinline__ void mid_unpack(uint64_t w, svd2_mid<double> &m)
{
    const uint32_t b = (uint32_t)w;
    m.t = b & 15; m.tp = (b >> 4) & 15; m.flags = (b >> 8) & 255;
    m.c15 = (b >> 16) & 1; m.pu = (b >> 17) & 1; m.pv = (b >> 18) & 1; m.na = (b >> 19) & 1;
    m.nb = (b >> 20) & 1; m.n12 = (b >> 21) & 1; m.n22 = (b >> 22) & 1;
    m.s = (int)((uint32_t)(w >> 32) & 0xFFFF) - 32768;
}

// Phases 1-2.  Matrices finished here (the simple classes, the fallback, non-finite inputs)
// get their results; the others get the parked state.
template <bool NCR>
__global__ void __launch_bounds__(256, 8) svd2a_kernel(const svd_args<double> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const double g11 = __ldcs(a.g0 + i), g21 = __ldcs(a.g1 + i), g12 = __ldcs(a.g2 + i), g22 = __ldcs(a.g3 + i);
        svd2_out<double> o;
        svd2_mid<double> m;
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22)) {
            if (svd2_a<double, NCR, SPLIT_FDIV_A, SPLIT_FDIV_AT>(g11, g21, g12, g22, o, m)) {
                a.u0[i] = m.r11; a.u1[i] = m.r12; a.u2[i] = m.r22;
                if (m.c15) { a.u3[i] = m.tth; a.v0[i] = m.secth; }
                a.s1[i] = dfrom(mid_pack(m));
                continue;
            }
        } else {
            nan_out(o);
        }
        store_out(a, i, o);
    }
}

// Phase 3 for the matrices whose sigma1 plane holds a packed word (sign bit set).
template <bool NCR>
__global__ void __launch_bounds__(256, 8) svd2b_kernel(const svd_args<double> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const uint64_t w = dbits(a.s1[i]);
        if (!(w & D_SIGN)) continue;
        svd2_mid<double> m;
        mid_unpack(w, m);
        m.r11 = a.u0[i]; m.r12 = a.u1[i]; m.r22 = a.u2[i];
        if (m.c15) { m.tth = a.u3[i]; m.secth = a.v0[i]; }
        else { m.tth = 0.0; m.secth = 0.0; }
        svd2_out<double> o;
        svd2_b<double, SPLIT_FDIV_B, NCR>(m, o);
        store_out(a, i, o);
    }
}

// The split form: two launches over the whole batch, no allocation.
template <bool NCR>
static int launch_split(const svd_args<double> &a, cudaStream_t st)
{
    static thread_local int cdev = -1, cblocks_a = 0, cblocks_b = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cdev) {
        int na = 0, nb = 0;
        if (grid_for(svd2a_kernel<NCR>, 256, 0, &na) != 0) return K2SVD_ECUDA;
        if (grid_for(svd2b_kernel<NCR>, 256, 0, &nb) != 0) return K2SVD_ECUDA;
        cdev = dev; cblocks_a = na; cblocks_b = nb;
    }
    const int64_t need = (a.n + 255) / 256;
    svd2a_kernel<NCR><<<(int)(need < cblocks_a ? need : cblocks_a), 256, 0, st>>>(a);
    svd2b_kernel<NCR><<<(int)(need < cblocks_b ? need : cblocks_b), 256, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

// General matrices: the split form for double batches of SPLIT_MIN or more, the fused
// kernel for smaller ones (one launch), for float and for the variant with the hypot that is
// not correctly rounded.
template <typename T, bool NCR>
static int launch_general(const svd_args<T> &a, cudaStream_t st)
{
    if constexpr (sizeof(T) == 8 && !NCR) {
        if (a.n >= SPLIT_MIN) return launch_split<NCR>(a, st);
    }
    return launch<T, false, NCR>(a, st);
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
    return launch_general<T, NCR>(a, (cudaStream_t)stream);
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
