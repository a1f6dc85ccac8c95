// The batched 2x2 SVD kernel (arXiv 2407.13116, Sect. 3) and its host-side argument checks,
// shared by the translation units of the correctly rounded method (k2_gesvd2.cu) and of the
// variant with the hypot that is not correctly rounded (k2_ncr.cu).
//
// One matrix per thread.  Inputs and outputs are SoA planes, so every load and store of a
// warp touches 32 consecutive elements of one plane (fully coalesced).  The grid is
// persistent: (SM count) x (resident blocks per SM) blocks stride over the batch.
#pragma once
#include <cstdint>
#include <mutex>
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
// (svd2b_kernel) as two launches, the state between them (R, tan and sec of theta, the
// permutations and signs: svd2_mid) in a scratch buffer.  Same operations as the fused
// kernel, so the same bits.  Each launch runs part of the method's code, and matrices of
// classes 13 and 15 meet in one copy of Alg. 1 and 2 instead of diverging into two.
// Each half also gets its own placement of the quotients (SPLIT_FDIV_*).  Measured on a
// GB300 against the fused kernel: 22% faster on wide-range matrices (all of class 15), 32%
// faster on narrow-range ones with triangular and zero-row inputs mixed in.  For float the
// fused kernel stays faster (the split one took 1.38 times as long).
// ---------------------------------------------------------------------------------------
template <typename T> struct mid_planes {
    T *r11, *r12, *r22, *tth, *secth;
    int32_t *s, *bits;
};
// Which quotients use the FP64 divider (csdiv): the three of eq. (QR15) in phases 1-2, none
// in phase 3.  Phases 1-2 are integer-heavy (the hypots, eq. (EXT)) and phase 3 FP64-heavy,
// so the FP64 divider moves to the first half: on 2^26 wide-range matrices 19.1 ms against
// 24.1 ms with the fused kernel's placement (the cos/sin quotients of Alg. 1 and 2 on the
// divider), 20.0 with both, 20.3 with neither.
constexpr bool SPLIT_FDIV_A = true, SPLIT_FDIV_B = false;
// bits: t | t' << 4 | phase-1-2 flags << 8 | c15 << 16 | pu << 17 | pv << 18 | na << 19 |
// nb << 20 | n12 << 21 | n22 << 22 | MID_B (phase 3 still to run)
constexpr int32_t MID_B = 1 << 23;

template <typename T, bool NCR>
__global__ void __launch_bounds__(256, 8) svd2a_kernel(const svd_args<T> a, const mid_planes<T> mp)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const T g11 = __ldcs(a.g0 + i), g21 = __ldcs(a.g1 + i), g12 = __ldcs(a.g2 + i), g22 = __ldcs(a.g3 + i);
        svd2_out<T> o;
        svd2_mid<T> m;
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22)) {
            if (svd2_a<T, NCR, SPLIT_FDIV_A>(g11, g21, g12, g22, o, m)) {
                mp.r11[i] = m.r11; mp.r12[i] = m.r12; mp.r22[i] = m.r22;
                if (m.c15) { mp.tth[i] = m.tth; mp.secth[i] = m.secth; }
                mp.s[i] = m.s;
                mp.bits[i] = m.t | (m.tp << 4) | (m.flags << 8) | (m.c15 << 16) | (m.pu << 17) | (m.pv << 18) |
                             (m.na << 19) | (m.nb << 20) | (m.n12 << 21) | (m.n22 << 22) | MID_B;
                continue;
            }
        } else {
            nan_out(o);
        }
        mp.bits[i] = 0;
        store_out(a, i, o);
    }
}

template <typename T, bool NCR>
__global__ void __launch_bounds__(256, 8) svd2b_kernel(const svd_args<T> a, const mid_planes<T> mp)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const int32_t b = __ldcs(mp.bits + i);
        if (!(b & MID_B)) continue;
        svd2_mid<T> m;
        m.t = b & 15; m.tp = (b >> 4) & 15; m.flags = (b >> 8) & 255;
        m.c15 = (b >> 16) & 1; m.pu = (b >> 17) & 1; m.pv = (b >> 18) & 1; m.na = (b >> 19) & 1;
        m.nb = (b >> 20) & 1; m.n12 = (b >> 21) & 1; m.n22 = (b >> 22) & 1;
        m.s = __ldcs(mp.s + i);
        m.r11 = __ldcs(mp.r11 + i); m.r12 = __ldcs(mp.r12 + i); m.r22 = __ldcs(mp.r22 + i);
        if (m.c15) { m.tth = __ldcs(mp.tth + i); m.secth = __ldcs(mp.secth + i); }
        else { m.tth = T(0); m.secth = T(0); }
        svd2_out<T> o;
        svd2_b<T, SPLIT_FDIV_B, NCR>(m, o);
        store_out(a, i, o);
    }
}

// A private stream-ordered memory pool per device for the split form's scratch: allocations
// are ordered on the caller's stream (safe for concurrent calls on several streams) and the
// pool keeps up to SPLIT_KEEP bytes between calls.
constexpr int64_t SPLIT_CHUNK = 1 << 24;                  // matrices per pair of launches
constexpr int64_t SPLIT_MIN = 1 << 16;                    // smaller batches: the fused kernel
constexpr uint64_t SPLIT_KEEP = 1ull << 30;

static cudaMemPool_t split_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!pools[dev]) {
        cudaMemPoolProps pp = {};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        cudaMemPool_t p;
        if (cudaMemPoolCreate(&p, &pp) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        uint64_t keep = SPLIT_KEEP;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

template <typename T> static svd_args<T> shifted(const svd_args<T> &a, int64_t off, int64_t len)
{
    svd_args<T> b = a;
    b.g0 += off; b.g1 += off; b.g2 += off; b.g3 += off;
    b.u0 += off; b.u1 += off; b.u2 += off; b.u3 += off;
    b.v0 += off; b.v1 += off; b.v2 += off; b.v3 += off;
    b.s1 += off; b.s2 += off;
    if (b.se1) { b.se1 += off; b.se2 += off; }
    if (b.sf1) { b.sf1 += off; b.sf2 += off; }
    if (b.info) b.info += off;
    b.n = len;
    return b;
}

// The split form (falls back to the fused kernel when no scratch can be had).
template <typename T, bool NCR>
static int launch_split(const svd_args<T> &a, cudaStream_t st)
{
    static thread_local int cdev = -1, cblocks_a = 0, cblocks_b = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cdev) {
        int na = 0, nb = 0;
        if (grid_for(svd2a_kernel<T, NCR>, 256, 0, &na) != 0) return K2SVD_ECUDA;
        if (grid_for(svd2b_kernel<T, NCR>, 256, 0, &nb) != 0) return K2SVD_ECUDA;
        cdev = dev; cblocks_a = na; cblocks_b = nb;
    }
    const int64_t chunk = a.n < SPLIT_CHUNK ? a.n : SPLIT_CHUNK;
    const size_t bytes = (size_t)chunk * (5 * sizeof(T) + 2 * sizeof(int32_t));
    cudaMemPool_t pool = split_pool(dev);
    void *ws = nullptr;
    if (!pool || cudaMallocFromPoolAsync(&ws, bytes, pool, st) != cudaSuccess) {
        cudaGetLastError();                                   // no scratch: the fused kernel
        return launch<T, false, NCR>(a, st);
    }
    mid_planes<T> mp;
    T *tp = (T *)ws;
    mp.r11 = tp; mp.r12 = tp + chunk; mp.r22 = tp + 2 * chunk; mp.tth = tp + 3 * chunk; mp.secth = tp + 4 * chunk;
    mp.s = (int32_t *)(tp + 5 * chunk); mp.bits = mp.s + chunk;
    for (int64_t off = 0; off < a.n; off += chunk) {
        const int64_t len = (a.n - off) < chunk ? (a.n - off) : chunk;
        const svd_args<T> b = shifted(a, off, len);
        const int64_t need = (len + 255) / 256;
        svd2a_kernel<T, NCR><<<(int)(need < cblocks_a ? need : cblocks_a), 256, 0, st>>>(b, mp);
        svd2b_kernel<T, NCR><<<(int)(need < cblocks_b ? need : cblocks_b), 256, 0, st>>>(b, mp);
    }
    const cudaError_t e = cudaPeekAtLastError();
    cudaFreeAsync(ws, st);
    return e == cudaSuccess ? 0 : K2SVD_ECUDA;
}

// General matrices: the split form for double batches of SPLIT_MIN or more, the fused
// kernel for smaller ones (one launch, no scratch), for float and for the variant with the
// hypot that is not correctly rounded.
template <typename T, bool NCR>
static int launch_general(const svd_args<T> &a, cudaStream_t st)
{
    if constexpr (sizeof(T) == 8 && !NCR) {
        if (a.n >= SPLIT_MIN) return launch_split<T, NCR>(a, st);
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
