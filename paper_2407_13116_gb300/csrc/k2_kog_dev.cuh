// Device parts of the batched n x n Kogbetliantz SVD (eq. (SVD), Sect. 1): the parallel
// modulus strategy, the rotations, the deterministic norms, and the per-matrix phases used
// by both the persistent kernel and the per-step kernels.
#pragma once
#include <climits>
#include <cstdint>

#include "k2_svd2.cuh"

namespace k2 {

// One matrix of a batch.  G scratch (goff) is used when G does not live in shared memory.
struct kog_desc {
    int32_t n, idx;       // order, index in the caller's batch
    int64_t off, soff;    // element offsets of A/U/V and of S
    int64_t goff;         // element offset of this matrix's scratch in the workspace: G when
                          // it is not in shared memory, then (dynamic ordering) the weights
};

// Pair p of step k of the modulus strategy: the pairs i < j with i + j = k (mod n), in
// increasing i: first i = 0 .. ceil(k/2)-1 with j = k - i, then i = k+1 .. with j = k + n - i.
__device__ __forceinline__ int modulus_count(int n, int k) { return ((k + 1) >> 1) + ((n - k - 1) >> 1); }
__device__ __forceinline__ void modulus_pair(int n, int k, int p, int &i, int &j)
{
    const int c1 = (k + 1) >> 1;
    if (p < c1) { i = p; j = k - p; }
    else { i = k + 1 + (p - c1); j = k + n - i; }
}

// The indices left unpaired by step k (2i = k mod n): one when n is odd, two when n and k
// are even, none otherwise; s = 0, 1 selects which.
__device__ __forceinline__ int modulus_single(int n, int k, int s)
{
    if (n & 1) return (k & 1) ? (k + n) >> 1 : k >> 1;
    return (k >> 1) + s * (n >> 1);
}

// Group of index r in step k: returns its pair's index p (with modulus_pair(n, k, p) = (i, j))
// or -1 when r is unpaired (then i = j = r).
__device__ __forceinline__ int modulus_group(int n, int k, int r, int &i, int &j)
{
    int q = k - r;
    if (q < 0) q += n;                                  // partner: r + q = k (mod n)
    if (q == r) { i = j = r; return -1; }
    i = min(r, q); j = max(r, q);
    return (i + j == k) ? i : ((k + 1) >> 1) + (i - k - 1);
}

// (x, y) <- (fma(m21, y, m11 x), fma(m22, y, m12 x)), m column-major (m11, m21, m12, m22)
// with its elements ps apart
template <typename T>
__device__ __forceinline__ void rot2(T &x, T &y, const T *m, int ps = 1)
{
    const T a = x, b = y;
    x = fma(m[ps], b, m[0] * a);
    y = fma(m[3 * ps], b, m[2 * ps] * a);
}

template <typename T> struct kog_eps;
template <> struct kog_eps<double> { __device__ static double v() { return 0x1p-52; } };
template <> struct kog_eps<float> { __device__ static float v() { return 0x1p-23f; } };

// Pivot SVD of [[a, b], [c, d]] (g11 = a, g21 = c, g12 = b, g22 = d) into the ten values
// m[0], m[ps], ..., m[9 ps]: U-hat (4, column-major, -0 as +0), V-hat (4), sigma1, sigma2
// (rounded).
template <typename T>
__device__ __forceinline__ void kog_pivot(T g11, T g21, T g12, T g22, T *m, int ps = 1)
{
    svd2_out<T> o;
    svd2<T>(g11, g21, g12, g22, o);
    m[0] = unneg0(o.U.a11); m[ps] = unneg0(o.U.a21); m[2 * ps] = unneg0(o.U.a12); m[3 * ps] = unneg0(o.U.a22);
    m[4 * ps] = unneg0(o.V.a11); m[5 * ps] = unneg0(o.V.a21); m[6 * ps] = unneg0(o.V.a12); m[7 * ps] = unneg0(o.V.a22);
    m[8 * ps] = ef_fl(o.s1);
    m[9 * ps] = ef_fl(o.s2);
}

// Block-level helpers.  All threads of the block (or the group running one matrix) call
// them; `scratch` is shared memory for n values of T plus a few words.
// sqrt of the column-sum-ordered sum of squares (diagonal skipped when off_only).
template <typename T>
__device__ __forceinline__ T kog_norm(const T *G, int n, int ld, bool off_only, T *colsum, T *bcast)
{
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        T s = T(0);
        const T *col = G + (size_t)c * ld;
        for (int r = 0; r < n; ++r)
            if (!off_only || r != c) s = fma(col[r], col[r], s);
        colsum[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T tot = T(0);
        for (int c = 0; c < n; ++c) tot = tot + colsum[c];
        *bcast = sqrt(tot);
    }
    __syncthreads();
    T r = *bcast;
    __syncthreads();
    return r;
}

}  // namespace k2
