// Batched 2x2 SVD kernels (arXiv 2407.13116, Sect. 3) and their C-ABI entry points
// k2svd_{d,s}gesvd2 and k2svd_{d,s}trsvd2, plus phase 1 alone (k2svd_{d,s}prescale2) and
// the xLASV2 argument shape (k2svd_{d,s}lasv2), declared in include/k2svd.h.
//
// One matrix per thread.  Inputs and outputs are SoA planes, so every load and store of a
// warp touches 32 consecutive elements of one plane (fully coalesced).  The grid is
// persistent: (SM count) x (resident blocks per SM) blocks stride over the batch.
#include <climits>
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

// At most 64 registers a thread, so 8 blocks (32 warps) are resident per SM: 5% faster than
// the unconstrained 80-register build for FP64 on a GB300.
template <typename T, bool TRI>
__global__ void __launch_bounds__(128, 8) svd2_kernel(const svd_args<T> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const T g11 = a.g0[i];
        const T g21 = TRI ? T(0) : a.g1[i];
        const T g12 = a.g2[i];
        const T g22 = a.g3[i];
        svd2_out<T> o;
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22)) {
            svd2<T, !TRI>(g11, g21, g12, g22, o);              // general matrices leave the FP64 pipe room
        } else {
            const T qn = T(NAN);
            o.U.a11 = o.U.a21 = o.U.a12 = o.U.a22 = qn;
            o.V.a11 = o.V.a21 = o.V.a12 = o.V.a22 = qn;
            o.s1.e = o.s2.e = 0; o.s1.f = o.s2.f = qn;
            o.info = -1;
        }
        a.u0[i] = pz(o.U.a11); a.u1[i] = pz(o.U.a21); a.u2[i] = pz(o.U.a12); a.u3[i] = pz(o.U.a22);
        a.v0[i] = pz(o.V.a11); a.v1[i] = pz(o.V.a21); a.v2[i] = pz(o.V.a12); a.v3[i] = pz(o.V.a22);
        if (o.info >= 0) {
            a.s1[i] = ef_fl(o.s1); a.s2[i] = ef_fl(o.s2);
        } else {
            a.s1[i] = o.s1.f; a.s2[i] = o.s2.f;
        }
        if (a.se1) { a.se1[i] = o.s1.e; a.se2[i] = o.s2.e; }
        if (a.sf1) { a.sf1[i] = o.s1.f; a.sf2[i] = o.s2.f; }
        if (a.info) a.info[i] = o.info;
    }
}

template <typename T, bool TRI>
static int launch(const svd_args<T> &a, cudaStream_t st)
{
    static thread_local int cached_dev = -1, cached_blocks = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    if (dev != cached_dev) {
        int nb = 0;
        if (grid_for(svd2_kernel<T, TRI>, 128, 0, &nb) != 0) return K2SVD_ECUDA;
        cached_dev = dev; cached_blocks = nb;
    }
    int64_t need = (a.n + 127) / 128;
    int blocks = (int)(need < cached_blocks ? need : cached_blocks);
    svd2_kernel<T, TRI><<<blocks, 128, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

template <typename T>
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
    return launch<T, false>(a, (cudaStream_t)stream);
}

template <typename T>
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
    return launch<T, true>(a, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------
// Phase 1 alone: Gs = 2^s G (Sect. 3.1) with the scale type raised by `extra`.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) prescale_kernel(const T *g0, const T *g1, const T *g2, const T *g3, T *o0,
                                                       T *o1, T *o2, T *o3, int32_t *sv, int32_t *types, int extra,
                                                       int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T g11 = g0[i], g21 = g1[i], g12 = g2[i], g22 = g3[i];
        int t = -1, sc = 0, tp = 0;
        if (is_fin(g11) && is_fin(g21) && is_fin(g12) && is_fin(g22)) phase1(g11, g21, g12, g22, extra, t, sc, tp);
        o0[i] = g11; o1[i] = g21; o2[i] = g12; o3[i] = g22;
        sv[i] = sc;
        if (types) types[i] = t < 0 ? -1 : (t | (tp << 4));
    }
}

// ---------------------------------------------------------------------------------------
// The xLASV2 argument shape: R = [[F, G], [0, H]] by the method, re-expressed as signed
// singular values and two rotations (first columns of U and V; the sign of SSMIN is
// det(U) det(V), read from the exact structure of U and V: a rotation has u22 = u11 and
// u12 = -u21, a reflection u22 = -u11 and u12 = u21).
// ---------------------------------------------------------------------------------------
// x == y for non-NaN values (+0 and -0 equal), on the bit patterns
__device__ __forceinline__ bool same_val(double x, double y) { return dbits(unneg0(x)) == dbits(unneg0(y)); }
__device__ __forceinline__ bool same_val(float x, float y) { return fbits(unneg0(x)) == fbits(unneg0(y)); }

template <typename T>
__global__ void __launch_bounds__(128, 8) lasv2_kernel(const T *F, const T *Gp, const T *H, T *ssmin, T *ssmax,
                                                       T *snr, T *csr, T *snl, T *csl, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T f = F[i], g = Gp[i], h = H[i];
        if (!(is_fin(f) && is_fin(g) && is_fin(h))) {
            const T qn = T(NAN);
            ssmin[i] = ssmax[i] = snr[i] = csr[i] = snl[i] = csl[i] = qn;
            continue;
        }
        svd2_out<T> o;
        svd2<T>(f, T(0), g, h, o);
        const bool ru = same_val(o.U.a22, o.U.a11) && same_val(o.U.a12, ngt(o.U.a21));
        const bool rv = same_val(o.V.a22, o.V.a11) && same_val(o.V.a12, ngt(o.V.a21));
        const T s1 = ef_fl(o.s1), s2 = ef_fl(o.s2);
        ssmax[i] = s1;
        ssmin[i] = unneg0(ru == rv ? s2 : ngt(s2));
        csl[i] = unneg0(o.U.a11); snl[i] = unneg0(o.U.a21);
        csr[i] = unneg0(o.V.a11); snr[i] = unneg0(o.V.a21);
    }
}

template <typename K>
static int grid_cached(K kernel, int threads, int *cache_dev, int *cache_blocks)
{
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (dev != *cache_dev) {
        int nb = 0;
        if (grid_for(kernel, threads, 0, &nb) != 0) return -1;
        *cache_dev = dev; *cache_blocks = nb;
    }
    return *cache_blocks;
}

template <typename T>
static int prescale2(int64_t n, const T *G, int64_t ldg, T *Gs, int64_t ldgs, int32_t *s, int32_t *types,
                     int32_t extra, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!G) return -2;
    if (ldg < n) return -3;
    if (!Gs) return -4;
    if (ldgs < n) return -5;
    if (!s) return -6;
    if (extra < 0 || extra > 64) return -8;
    static thread_local int cdev = -1, cblocks = 0;
    int nb = grid_cached(prescale_kernel<T>, 256, &cdev, &cblocks);
    if (nb < 0) return K2SVD_ECUDA;
    int64_t need = (n + 255) / 256;
    int blocks = (int)(need < nb ? need : nb);
    prescale_kernel<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(G, G + ldg, G + 2 * ldg, G + 3 * ldg, Gs, Gs + ldgs,
                                                                  Gs + 2 * ldgs, Gs + 3 * ldgs, s, types, extra, n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

template <typename T>
static int lasv2(int64_t n, const T *F, const T *Gp, const T *H, T *ssmin, T *ssmax, T *snr, T *csr, T *snl, T *csl,
                 void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!F) return -2;
    if (!Gp) return -3;
    if (!H) return -4;
    if (!ssmin) return -5;
    if (!ssmax) return -6;
    if (!snr) return -7;
    if (!csr) return -8;
    if (!snl) return -9;
    if (!csl) return -10;
    static thread_local int cdev = -1, cblocks = 0;
    int nb = grid_cached(lasv2_kernel<T>, 128, &cdev, &cblocks);
    if (nb < 0) return K2SVD_ECUDA;
    int64_t need = (n + 127) / 128;
    int blocks = (int)(need < nb ? need : nb);
    lasv2_kernel<T><<<blocks, 128, 0, (cudaStream_t)stream>>>(F, Gp, H, ssmin, ssmax, snr, csr, snl, csl, n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

}  // namespace k2

extern "C" {

int k2svd_dprescale2(int64_t batch, const double *G, int64_t ldg, double *Gs, int64_t ldgs, int32_t *s,
                     int32_t *types, int32_t extra, void *stream)
{
    return k2::prescale2<double>(batch, G, ldg, Gs, ldgs, s, types, extra, stream);
}

int k2svd_sprescale2(int64_t batch, const float *G, int64_t ldg, float *Gs, int64_t ldgs, int32_t *s,
                     int32_t *types, int32_t extra, void *stream)
{
    return k2::prescale2<float>(batch, G, ldg, Gs, ldgs, s, types, extra, stream);
}

int k2svd_dlasv2(int64_t batch, const double *F, const double *G, const double *H, double *ssmin, double *ssmax,
                 double *snr, double *csr, double *snl, double *csl, void *stream)
{
    return k2::lasv2<double>(batch, F, G, H, ssmin, ssmax, snr, csr, snl, csl, stream);
}

int k2svd_slasv2(int64_t batch, const float *F, const float *G, const float *H, float *ssmin, float *ssmax,
                 float *snr, float *csr, float *snl, float *csl, void *stream)
{
    return k2::lasv2<float>(batch, F, G, H, ssmin, ssmax, snr, csr, snl, csl, stream);
}


int k2svd_dgesvd2(int64_t batch, const double *G, int64_t ldg, double *U, int64_t ldu, double *V, int64_t ldv,
                  double *S, int64_t lds, int32_t *Se, double *Sf, int32_t *info, void *stream)
{
    return k2::gesvd2<double>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_sgesvd2(int64_t batch, const float *G, int64_t ldg, float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info, void *stream)
{
    return k2::gesvd2<float>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_dtrsvd2(int64_t batch, const double *F, const double *Gu, const double *H, double *U, int64_t ldu,
                  double *V, int64_t ldv, double *S, int64_t lds, int32_t *Se, double *Sf, int32_t *info,
                  void *stream)
{
    return k2::trsvd2<double>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_strsvd2(int64_t batch, const float *F, const float *Gu, const float *H, float *U, int64_t ldu,
                  float *V, int64_t ldv, float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info,
                  void *stream)
{
    return k2::trsvd2<float>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_version(void) { return 100; }

}  // extern "C"
