/*
 * k2probe -- pipe-throughput probes used to measure the roofline denominators of the
 * libk2svd kernels on the device at hand.  They are measurement helpers, not part of the
 * method; the paper has no counterpart.
 *
 * k2probe_rate: runs a fixed arithmetic loop of one operation kind on every SM and returns
 * the sustained rate in operations per second in *rate.  Enough independent chains are in
 * flight per thread to hide latency, so the result is the issue-limited throughput.
 *   op   0 = FP64 fma, 1 = FP64 division, 2 = FP64 square root,
 *        3 = FP32 fma, 4 = FP32 division, 5 = FP32 square root
 *   rate host pointer, receives operations per second
 * Returns 0, -1 for an unknown op, K2SVD_ECUDA (-1000) when a CUDA call failed.  Allocates
 * and frees a small device buffer; synchronizes the device.
 */
#ifndef K2PROBE_H
#define K2PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int k2probe_rate(int op, double *rate);

/*
 * k2probe_div / k2probe_hypot -- elementwise checks of two primitives of the 2x2 kernels on
 * device arrays of n doubles: q[i] = a[i] / b[i] by the integer-pipe correctly rounded
 * division, h[i] = hypot(a[i], b[i]) by the correctly rounded hypot (Sect. 2).  For testing
 * these primitives against the FP64 divider and an exact reference; not part of the method.
 * Returns 0, -1 (n < 0), -2 (null pointer), -1000 (a CUDA launch error).  Asynchronous on
 * `stream`.
 */
int k2probe_div(int64_t n, const double *a, const double *b, double *q, void *stream);
int k2probe_hypot(int64_t n, const double *a, const double *b, double *h, void *stream);
/* k2probe_hypotf -- the binary32 correctly rounded hypot, same conventions. */
int k2probe_hypotf(int64_t n, const float *a, const float *b, float *h, void *stream);
/* k2probe_hypot_ncr / k2probe_hypotf_ncr -- the hypot that is not correctly rounded, used by
 * the k2svd_?gesvd2_ncr variant (Alg. 1's branch for such a hypot): xLAPY2's scaled formula
 * w * sqrt(fma(q, q, 1)), q = z / w, w = max(|a|,|b|), z = min(|a|,|b|), each step rounded to
 * nearest; +Inf if an argument is infinite, else NaN if one is NaN.  Same conventions. */
int k2probe_hypot_ncr(int64_t n, const double *a, const double *b, double *h, void *stream);
int k2probe_hypotf_ncr(int64_t n, const float *a, const float *b, float *h, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* K2PROBE_H */
