// Batched 2x2 SVD entry points (arXiv 2407.13116, Sect. 3) k2svd_{d,s}gesvd2 and
// k2svd_{d,s}trsvd2 (kernel in k2_svd2_kernel.cuh), plus phase 1 alone (k2svd_{d,s}prescale2)
// and the xLASV2 argument shape (k2svd_{d,s}lasv2), declared in include/k2svd.h.
//
// One matrix per thread, SoA planes (coalesced), persistent grids.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "k2_svd2_kernel.cuh"

namespace k2 {

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

// Full occupancy (8 blocks of 256, 32 registers) as in svd2_kernel: 7% faster than 64 registers.
template <typename T>
__global__ void __launch_bounds__(256, 8) lasv2_kernel(const T *F, const T *Gp, const T *H, T *ssmin, T *ssmax,
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
    int nb = grid_cached(lasv2_kernel<T>, 256, &cdev, &cblocks);
    if (nb < 0) return K2SVD_ECUDA;
    int64_t need = (n + 127) / 128;
    int blocks = (int)(need < nb ? need : nb);
    lasv2_kernel<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(F, Gp, H, ssmin, ssmax, snr, csr, snl, csl, n);
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
    return k2::gesvd2<double, false>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_sgesvd2(int64_t batch, const float *G, int64_t ldg, float *U, int64_t ldu, float *V, int64_t ldv,
                  float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info, void *stream)
{
    return k2::gesvd2<float, false>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_dtrsvd2(int64_t batch, const double *F, const double *Gu, const double *H, double *U, int64_t ldu,
                  double *V, int64_t ldv, double *S, int64_t lds, int32_t *Se, double *Sf, int32_t *info,
                  void *stream)
{
    return k2::trsvd2<double, false>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_strsvd2(int64_t batch, const float *F, const float *Gu, const float *H, float *U, int64_t ldu,
                  float *V, int64_t ldv, float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info,
                  void *stream)
{
    return k2::trsvd2<float, false>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_version(void) { return 100; }

}  // extern "C"
