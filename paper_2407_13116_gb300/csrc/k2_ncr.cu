// The batched 2x2 SVD with a hypot that is not correctly rounded (arXiv 2407.13116, Alg. 1:
// the branch that computes tan(2 phi) without squaring when hypot is not correctly rounded,
// and that hypot everywhere the method calls one).  C-ABI entry points
// k2svd_{d,s}gesvd2_ncr and k2svd_{d,s}trsvd2_ncr, declared in include/k2svd.h.  Same kernel
// as the correctly rounded method (k2_svd2_kernel.cuh), instantiated with NCR = true.
#include "k2_svd2_kernel.cuh"

extern "C" {

int k2svd_dgesvd2_ncr(int64_t batch, const double *G, int64_t ldg, double *U, int64_t ldu, double *V, int64_t ldv,
                      double *S, int64_t lds, int32_t *Se, double *Sf, int32_t *info, void *stream)
{
    return k2::gesvd2<double, true>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_sgesvd2_ncr(int64_t batch, const float *G, int64_t ldg, float *U, int64_t ldu, float *V, int64_t ldv,
                      float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info, void *stream)
{
    return k2::gesvd2<float, true>(batch, G, ldg, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_dtrsvd2_ncr(int64_t batch, const double *F, const double *Gu, const double *H, double *U, int64_t ldu,
                      double *V, int64_t ldv, double *S, int64_t lds, int32_t *Se, double *Sf, int32_t *info,
                      void *stream)
{
    return k2::trsvd2<double, true>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

int k2svd_strsvd2_ncr(int64_t batch, const float *F, const float *Gu, const float *H, float *U, int64_t ldu,
                      float *V, int64_t ldv, float *S, int64_t lds, int32_t *Se, float *Sf, int32_t *info,
                      void *stream)
{
    return k2::trsvd2<float, true>(batch, F, Gu, H, U, ldu, V, ldv, S, lds, Se, Sf, info, stream);
}

}  // extern "C"
