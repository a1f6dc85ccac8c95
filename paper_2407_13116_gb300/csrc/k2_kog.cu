// Batched n x n Kogbetliantz SVD (eq. (SVD) of Sect. 1) with the 2x2 method of Sect. 3 as
// the pivot solver: k2svd_{d,s}kogbet, k2svd_{d,s}kogbet_ws, k2svd_{d,s}kog_sigma_bwd
// (include/k2svd.h).
//
// Persistent form: the matrices are grouped by order into buckets.  Each bucket is one
// persistent launch: every CTA takes the next matrix from a queue (largest first) and runs
// all of its sweeps alone, with G in shared memory (orders up to 128 double / 224 float)
// or in the workspace.  A step k is two phases separated by block barriers:
//   1. G <- U-hat^T G V-hat: every thread takes 2x2 blocks (rows of one pivot pair or
//      unpaired index, columns of another) and applies the row rotation, then the column
//      rotation -- the same operations, in the same order, as rotating all rows first and
//      all columns second; diagonal pivot blocks become diag(sigma1, sigma2);
//   2. the U and V updates of step k.
// The pivot SVDs of step k+1 overlap both: before phase 1, the pivot threads (the first
// warps, one thread per pivot) compute the four elements of their pivot in G_{k+1} from
// G_k and the rotations of step k -- the same operations phase 1 applies to them -- and
// after a barrier they run the SVDs while the remaining warps do phases 1 and 2.  The long
// serial 2x2 SVDs thus hide behind the FP64 rotation work.  Blocks too small to spare a
// warp run the phases one after the other.  The pivot parameters are double buffered and
// stored by parameter (stride nmax/2+1), so a warp reads them without bank conflicts.
// The off-norm is summed column by column in a fixed order, so the sweep count -- and
// every bit of the result -- does not depend on the launch shape.
//
// Per-step form (K2SVD_KOG_PLAIN): G in the workspace, three launches per step over the
// whole batch, and a host read-back per sweep for the convergence test.
//
// Dynamic ordering (K2SVD_KOG_DYNAMIC, persistent form only): the pairs of a step are not
// the modulus strategy's but the greedy choice by decreasing weight w_ij = g_ji^2 + g_ij^2
// (Sect. 1 names the dynamic ordering as a candidate strategy); a step is then weights,
// selection, pivot SVDs and rotations one after the other (kog_dynamic).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "k2_kog_dev.cuh"
#include "k2svd.h"
#include "k2_launch.h"

namespace k2 {

// ---------------------------------------------------------------------------------------
// parameters and shared-memory layout
// ---------------------------------------------------------------------------------------
template <typename T> struct kog_params {
    const kog_desc *desc;
    int count;             // matrices in this launch
    int *queue;            // work counter (persistent) / per-matrix flags (per-step)
    const T *A;
    T *U, *V, *S;
    int32_t *sweeps, *info;
    T *gws;                // scratch base: G outside shared memory, pair weights
    int max_sweeps;
    double tol_factor;
    int nmax;              // largest order of the launch (shared-memory capacity)
    int wsm;               // dynamic ordering: the pair weights in shared memory (else after G)
};

// pivot parameters of one step: 10 values for each of at most nmax/2 pivots, stored by
// parameter with stride kog_piv_stride; two such buffers
__host__ __device__ constexpr int kog_piv_stride(int nmax) { return nmax / 2 + 1; }
template <typename T> __host__ __device__ constexpr size_t kog_piv_elems(int nmax) { return (size_t)kog_piv_stride(nmax) * 10; }

// Shared memory of the persistent kernel: G (unless in the workspace), two buffers of pivot
// parameters, the column sums (nmax), perm and flip (2 nmax ints), then U and V (nmax^2 each)
// when they are staged in shared memory too (uvs).
template <typename T>
__host__ __device__ inline size_t kog_smem_bytes(int nmax, bool gg, bool uvs = false)
{
    size_t g = gg ? 0 : (size_t)(nmax + 1) * nmax * sizeof(T);
    size_t uv = uvs ? 2 * (size_t)nmax * nmax * sizeof(T) : 0;
    return g + 2 * kog_piv_elems<T>(nmax) * sizeof(T) + (size_t)nmax * sizeof(T) + 2 * (size_t)nmax * sizeof(int) + uv +
           64;
}
// U and V are staged in shared memory for orders up to KOG_UVS_MAX: the whole factorization
// then runs in shared memory and they are written out once, permuted, at the end.  Measured
// on the 8192-matrix workload (orders 8..128): the orders-8..32 bucket 9.35 ms against 9.68
// with U and V in global memory; staging up to order 48 or 64 made those buckets slower
// (33..64: 73.7 ms against 70.6 at 64), as the extra shared memory leaves fewer CTAs per SM
// for steps that wait on their pivot SVDs.
constexpr int KOG_UVS_MAX = 32;

// ---------------------------------------------------------------------------------------
// per-matrix phases shared by both forms (called by all threads of a block)
// ---------------------------------------------------------------------------------------
struct kog_sh {                       // block-shared scalars
    int slot, kmax, bad, uv;
    double b;
};

// Load A into G (leading dimension ld), U = V = I; returns the prescaling exponent k, or
// INT_MIN when A has a non-finite element (outputs set to NaN, info -1).
template <typename T>
__device__ int kog_load(const T *A, T *G, int ld, T *U, T *V, int n, kog_sh *sh)
{
    if (threadIdx.x == 0) { sh->kmax = INT_MIN; sh->bad = 0; }
    __syncthreads();
    int lmax = INT_MIN, bad = 0;
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int r = e % n, c = e / n;
        const T x = A[e];
        if (!isfinite(x)) bad = 1;
        else if (x != T(0)) lmax = max(lmax, fpt<T>::expo(x));
        G[(size_t)c * ld + r] = x;
        U[e] = (r == c) ? T(1) : T(0);
        V[e] = (r == c) ? T(1) : T(0);
    }
    if (lmax != INT_MIN) atomicMax(&sh->kmax, lmax);
    if (bad) atomicOr(&sh->bad, 1);
    __syncthreads();
    const int kmax = sh->kmax, isbad = sh->bad;
    __syncthreads();
    if (isbad) return INT_MIN;
    const int k = (kmax == INT_MIN) ? 0 : -(kmax + 1);
    if (k != 0)
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            T *g = &G[(size_t)(e / n) * ld + e % n];
            *g = fpt<T>::scale(*g, k);
        }
    __syncthreads();
    return k;
}

// Pivot SVDs of step st from G into piv (stride ps), by threads t0, t0+tn, ...
template <typename T>
__device__ __forceinline__ void kog_pivots(const T *G, int ld, int n, int st, T *piv, int ps, int t0, int tn)
{
    const int np = modulus_count(n, st);
    for (int p = t0; p < np; p += tn) {
        int i, j;
        modulus_pair(n, st, p, i, j);
        kog_pivot(G[(size_t)i * ld + i], G[(size_t)i * ld + j], G[(size_t)j * ld + i], G[(size_t)j * ld + j],
                  piv + p, ps);
    }
}

// Phase 1 of step st: G <- U-hat^T G V-hat by 2x2 blocks.  Block (a, b) has the rows of
// group a and the columns of group b, a group being a pivot pair (a < np) or an unpaired
// index.  Each element gets the row rotation first, then the column rotation.
template <typename T>
__device__ __forceinline__ void kog_g_item(T *G, int ld, int n, int st, int np, int nq, const T *piv, int ps, int w)
{
    const int a = w % nq, b = w / nq;
    int ia, ja = -1, ib, jb = -1;
    if (a < np) modulus_pair(n, st, a, ia, ja); else ia = modulus_single(n, st, a - np);
    if (b < np) modulus_pair(n, st, b, ib, jb); else ib = modulus_single(n, st, b - np);
    if (ja < 0 && jb < 0) return;                              // unpaired row and column
    if (a == b) {                                              // the pivot block -> diag(sigma)
        G[(size_t)ia * ld + ia] = piv[8 * ps + a];
        G[(size_t)ia * ld + ja] = T(0);
        G[(size_t)ja * ld + ia] = T(0);
        G[(size_t)ja * ld + ja] = piv[9 * ps + a];
        return;
    }
    T *c0 = G + (size_t)ib * ld, *c1 = jb >= 0 ? G + (size_t)jb * ld : nullptr;
    T x00 = c0[ia], x10 = T(0), x01 = T(0), x11 = T(0);
    if (ja >= 0) x10 = c0[ja];
    if (jb >= 0) { x01 = c1[ia]; if (ja >= 0) x11 = c1[ja]; }
    if (ja >= 0) {                                             // rows ia, ja <- U-hat^T
        rot2(x00, x10, piv + a, ps);
        if (jb >= 0) rot2(x01, x11, piv + a, ps);
    }
    if (jb >= 0) {                                             // columns ib, jb <- V-hat
        rot2(x00, x01, piv + 4 * ps + b, ps);
        if (ja >= 0) rot2(x10, x11, piv + 4 * ps + b, ps);
    }
    c0[ia] = x00;
    if (ja >= 0) c0[ja] = x10;
    if (jb >= 0) { c1[ia] = x01; if (ja >= 0) c1[ja] = x11; }
}

template <typename T>
__device__ __forceinline__ void kog_rotate_g(T *G, int ld, int n, int st, const T *piv, int ps, int t0, int tn)
{
    const int np = modulus_count(n, st), nq = n - np;          // groups: np pairs + (n - 2 np) singles
    const int items = nq * nq;
    for (int w = t0; w < items; w += tn) kog_g_item(G, ld, n, st, np, nq, piv, ps, w);
}

// U and V updates of step st (columns i, j of U <- U-hat, of V <- V-hat) by threads
// t0, t0+tn, ...  U and V live in global memory (L2), so each thread takes two items at a
// time and issues all eight loads before any arithmetic: the items touch distinct elements
// (the pairs of a step are disjoint), and two L2 round trips overlap instead of following
// one another.
template <typename T>
__device__ __forceinline__ void kog_rotate_uv(T *U, T *V, int n, int st, const T *piv, int ps, int t0, int tn)
{
    const int np = modulus_count(n, st);
    const int items = np * n;
    int w = t0;
    for (; w + tn < items; w += 2 * tn) {
        const int w1 = w + tn;
        const int r0 = w % n, p0 = w / n, r1 = w1 % n, p1 = w1 / n;
        int i0, j0, i1, j1;
        modulus_pair(n, st, p0, i0, j0);
        modulus_pair(n, st, p1, i1, j1);
        T *ua0 = U + (size_t)i0 * n + r0, *ub0 = U + (size_t)j0 * n + r0;
        T *va0 = V + (size_t)i0 * n + r0, *vb0 = V + (size_t)j0 * n + r0;
        T *ua1 = U + (size_t)i1 * n + r1, *ub1 = U + (size_t)j1 * n + r1;
        T *va1 = V + (size_t)i1 * n + r1, *vb1 = V + (size_t)j1 * n + r1;
        T x0 = *ua0, y0 = *ub0, s0 = *va0, t0v = *vb0, x1 = *ua1, y1 = *ub1, s1 = *va1, t1v = *vb1;
        rot2(x0, y0, piv + p0, ps);
        rot2(s0, t0v, piv + 4 * ps + p0, ps);
        rot2(x1, y1, piv + p1, ps);
        rot2(s1, t1v, piv + 4 * ps + p1, ps);
        *ua0 = x0; *ub0 = y0; *va0 = s0; *vb0 = t0v;
        *ua1 = x1; *ub1 = y1; *va1 = s1; *vb1 = t1v;
    }
    for (; w < items; w += tn) {
        const int r = w % n, p = w / n;
        int i, j;
        modulus_pair(n, st, p, i, j);
        rot2(U[(size_t)i * n + r], U[(size_t)j * n + r], piv + p, ps);
        rot2(V[(size_t)i * n + r], V[(size_t)j * n + r], piv + 4 * ps + p, ps);
    }
}

// The U and V updates of step st taken by whole warps from a shared work counter, 64 items
// at a time (two per lane, loads first as in kog_rotate_uv): warps that finish their other
// work early -- the pivot warps once their 2x2 SVDs are done -- take more of them.  Called by
// converged warps; *ctr is zero at the start of the step.
template <typename T>
__device__ __forceinline__ void kog_rotate_uv_dyn(T *U, T *V, int n, int st, const T *piv, int ps, int *ctr)
{
    const int np = modulus_count(n, st);
    const int items = np * n;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(ctr, 64);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= items) break;
        const int wa = base + lane, wb = base + 32 + lane;
        if (wb < items) {
            const int r0 = wa % n, p0 = wa / n, r1 = wb % n, p1 = wb / n;
            int i0, j0, i1, j1;
            modulus_pair(n, st, p0, i0, j0);
            modulus_pair(n, st, p1, i1, j1);
            T *ua0 = U + (size_t)i0 * n + r0, *ub0 = U + (size_t)j0 * n + r0;
            T *va0 = V + (size_t)i0 * n + r0, *vb0 = V + (size_t)j0 * n + r0;
            T *ua1 = U + (size_t)i1 * n + r1, *ub1 = U + (size_t)j1 * n + r1;
            T *va1 = V + (size_t)i1 * n + r1, *vb1 = V + (size_t)j1 * n + r1;
            T x0 = *ua0, y0 = *ub0, s0 = *va0, t0v = *vb0, x1 = *ua1, y1 = *ub1, s1 = *va1, t1v = *vb1;
            rot2(x0, y0, piv + p0, ps);
            rot2(s0, t0v, piv + 4 * ps + p0, ps);
            rot2(x1, y1, piv + p1, ps);
            rot2(s1, t1v, piv + 4 * ps + p1, ps);
            *ua0 = x0; *ub0 = y0; *va0 = s0; *vb0 = t0v;
            *ua1 = x1; *ub1 = y1; *va1 = s1; *vb1 = t1v;
        } else {
            for (int w = wa; w < items; w += 32) {
                const int r = w % n, p = w / n;
                int i, j;
                modulus_pair(n, st, p, i, j);
                rot2(U[(size_t)i * n + r], U[(size_t)j * n + r], piv + p, ps);
                rot2(V[(size_t)i * n + r], V[(size_t)j * n + r], piv + 4 * ps + p, ps);
            }
        }
    }
}

// Element (r, c) of G_{k+1} computed from G_k and the rotations of step st, with the
// operations phase 1 applies to it: the row rotation of r's pair (both columns of c's
// group), then the column rotation of c's pair; sigma or zero inside a pivot block.
template <typename T>
__device__ __forceinline__ T kog_next_entry(const T *G, int ld, int n, int st, const T *piv, int ps, int r, int c)
{
    int ia, ja, ib, jb;
    const int a = modulus_group(n, st, r, ia, ja), b = modulus_group(n, st, c, ib, jb);
    if (a >= 0 && a == b) return r == c ? piv[(r == ia ? 8 : 9) * ps + a] : T(0);
    auto g1 = [&](int x) -> T {                        // row-rotated element (r, x)
        if (a < 0) return G[(size_t)x * ld + r];
        const T u = G[(size_t)x * ld + ia], v = G[(size_t)x * ld + ja];
        return r == ia ? fma(piv[ps + a], v, piv[a] * u) : fma(piv[3 * ps + a], v, piv[2 * ps + a] * u);
    };
    if (b < 0) return g1(c);
    const T x = g1(ib), y = g1(jb);
    return c == ib ? fma(piv[5 * ps + b], y, piv[4 * ps + b] * x) : fma(piv[7 * ps + b], y, piv[6 * ps + b] * x);
}

// One step st of the persistent form (parameters in pc), leaving the pivot parameters of
// step nx in pn.  Ends with a block barrier.
template <typename T>
__device__ __forceinline__ void kog_step(T *G, int ld, T *U, T *V, int n, int st, int nx, const T *pc, T *pn, int ps,
                                         int *uvc)
{
    const int npn = modulus_count(n, nx);
    const int w0 = (npn + 31) & ~31;
    const int tid = threadIdx.x;
    if ((int)blockDim.x - w0 >= 32) {
        if (tid == 0) *uvc = 0;
        T g11 = T(0), g21 = T(0), g12 = T(0), g22 = T(0);
        if (tid < npn) {
            int i, j;
            modulus_pair(n, nx, tid, i, j);
            g11 = kog_next_entry(G, ld, n, st, pc, ps, i, i);
            g21 = kog_next_entry(G, ld, n, st, pc, ps, j, i);
            g12 = kog_next_entry(G, ld, n, st, pc, ps, i, j);
            g22 = kog_next_entry(G, ld, n, st, pc, ps, j, j);
        }
        __syncthreads();                                    // G_k read before phase 1 writes
        if (tid < w0) {
            if (tid < npn) kog_pivot(g11, g21, g12, g22, pn + tid, ps);
            __syncwarp();
        } else {
            kog_rotate_g(G, ld, n, st, pc, ps, tid - w0, blockDim.x - w0);
        }
        kog_rotate_uv_dyn(U, V, n, st, pc, ps, uvc);     // every warp, the pivot warps too
    } else {
        kog_rotate_g(G, ld, n, st, pc, ps, tid, blockDim.x);
        __syncthreads();
        kog_rotate_uv(U, V, n, st, pc, ps, tid, blockDim.x);
        kog_pivots(G, ld, n, nx, pn, ps, tid, blockDim.x);
    }
    __syncthreads();
}

// Sort the diagonal (descending, stable), write S, permute the columns of U and V through
// the staging area `stage` (n*n elements, may be G), or, when U and V were staged in shared
// memory (Us, Vs), straight from there into U and V.
template <typename T>
__device__ void kog_finish(const T *G, int ld, T *U, T *V, T *S, int n, int k, T *dg, int *perm, T *stage,
                           const T *Us = nullptr, const T *Vs = nullptr)
{
    // a negative diagonal element gives its sign to U's column (stored in the sign of dg's
    // slot as a flag array after the sort); |g_qq| are ranked
    int *flip = perm + n;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const T d = G[(size_t)q * ld + q];
        flip[q] = d < T(0);
        dg[q] = d < T(0) ? -d : d;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const T dq = dg[q];
        int rank = 0;
        for (int p = 0; p < n; ++p) {
            const T dp = dg[p];
            rank += (dp > dq) || (dp == dq && p < q);
        }
        perm[rank] = q;
        S[rank] = fpt<T>::scale(dq, -k);
    }
    __syncthreads();
    const int nn = n * n;
    for (int pass = 0; pass < 2; ++pass) {
        T *X = pass ? V : U;
        const T *from = pass ? Vs : Us;
        if (!from) {
            for (int e = threadIdx.x; e < nn; e += blockDim.x) stage[e] = X[e];
            __syncthreads();
            from = stage;
        }
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int src = perm[e / n];
            const T x = from[(size_t)src * n + e % n];
            X[e] = (pass == 0 && flip[src]) ? -x : x;
        }
        __syncthreads();
    }
}

template <typename T>
__device__ void kog_fail(T *U, T *V, T *S, int n)
{
    const T qn = T(NAN);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) { U[e] = qn; V[e] = qn; }
    for (int q = threadIdx.x; q < n; q += blockDim.x) S[q] = qn;
}

// ---------------------------------------------------------------------------------------
// persistent kernel
// ---------------------------------------------------------------------------------------
// MINB = 2 caps the registers at 64 a thread so that more CTAs share an SM: for buckets up
// to order 64, whose steps are bound by the latency of their pivot SVDs rather than by the
// FP64 rotations (order 64: 0.72 of the rotation floor against 0.65; order 128 and the
// whole 8192-matrix workload were slower with the cap).
template <typename T, bool GG, int MINB, bool UVS, int MAXT = 512>
__global__ void __launch_bounds__(MAXT, MINB) kog_persistent(const kog_params<T> P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ kog_sh sh;
    T *Gs = reinterpret_cast<T *>(smem);
    T *piv = Gs + (GG ? 0 : (size_t)(P.nmax + 1) * P.nmax);
    const int ps = kog_piv_stride(P.nmax);
    T *colsum = piv + 2 * kog_piv_elems<T>(P.nmax);
    int *perm = reinterpret_cast<int *>(colsum + P.nmax);
    T *Us = UVS ? reinterpret_cast<T *>(perm + 2 * P.nmax) : nullptr;
    T *Vs = UVS ? Us + (size_t)P.nmax * P.nmax : nullptr;
    for (;;) {
        if (threadIdx.x == 0) sh.slot = atomicAdd(P.queue, 1);
        __syncthreads();
        const int slot = sh.slot;
        __syncthreads();
        if (slot >= P.count) break;
        const kog_desc d = P.desc[slot];
        const int n = d.n, ld = GG ? n : n + 1;
        T *G = GG ? P.gws + d.goff : Gs;
        T *U = P.U + d.off, *V = P.V + d.off, *S = P.S + d.soff;
        T *Uw = UVS ? Us : U, *Vw = UVS ? Vs : V;        // where the sweeps update U and V
        const int k = kog_load(P.A + d.off, G, ld, Uw, Vw, n, &sh);
        if (k == INT_MIN) {
            kog_fail(U, V, S, n);
            if (threadIdx.x == 0) {
                if (P.sweeps) P.sweeps[d.idx] = 0;
                if (P.info) P.info[d.idx] = -1;
            }
            __syncthreads();
            continue;
        }
        T *bc = reinterpret_cast<T *>(&sh.b);
        const T nrm = kog_norm(G, n, ld, false, colsum, bc);
        const T tol = (T(P.tol_factor) * T(n)) * kog_eps<T>::v() * nrm;
        T off = kog_norm(G, n, ld, true, colsum, bc);
        int sw = 0;
        bool go = !(off < tol) && sw < P.max_sweeps && off > T(0);
        T *pc = piv, *pn = piv + kog_piv_elems<T>(P.nmax);
        if (go) {
            kog_pivots(G, ld, n, 0, pc, ps, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        while (go) {
            for (int st = 0; st < n; ++st) {
                // the pivots of the next step: step 0 of the next sweep after the last one
                // (unused when the sweeps end)
                kog_step(G, ld, Uw, Vw, n, st, st + 1 < n ? st + 1 : 0, pc, pn, ps, &sh.uv);
                T *t = pc; pc = pn; pn = t;
            }
            ++sw;
            off = kog_norm(G, n, ld, true, colsum, bc);
            go = !(off < tol) && sw < P.max_sweeps && off > T(0);
        }
        kog_finish(G, ld, U, V, S, n, k, colsum, perm, G, Us, Vs);
        if (threadIdx.x == 0) {
            if (P.sweeps) P.sweeps[d.idx] = sw;
            if (P.info) P.info[d.idx] = (off < tol || off == T(0)) ? 0 : 1;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// dynamic ordering: persistent kernel
// ---------------------------------------------------------------------------------------
// The greedy choice (scan the pairs by decreasing rank, take each whose indices are free)
// is computed as a matching of locally dominant pairs: in rounds, every free index finds its
// best free partner, and each pair of indices that are each other's best is taken.  Under a
// strict total order of the pairs (weight, then pair index) both give the same pairs -- the
// best remaining pair is always mutually best, and a mutually best pair is never beaten
// later by a pair sharing one of its indices -- while the rounds here are few (every round
// takes at least the best remaining pair) and each touches only the indices whose partner
// was just taken.
//
// Step k: (A) all threads rotate G with the pivots of step k (G becomes G_{k+1}); (B) while
// the last warps update U and V with step k's rotations, the first warps compute the
// weights of G_{k+1}, choose the pairs of step k+1 and run their pivot SVDs into the other
// buffer, so that the serial 2x2 SVDs hide behind the U and V work.
//
// Shared memory: G (unless GG), two buffers of pivot parameters, colsum (nmax), then ints:
// perm and flip (2 nmax, for kog_finish), two buffers of pairs pi, pj (nmax/2 + 1 each) and
// groups gi, gj (nmax each), used and best (nmax each), and four counters; then the
// n(n-1)/2 pair weights when they fit (P.wsm; in the workspace otherwise).  Rescanning a
// row of weights from global memory cost an L2 round trip per element: with the weights
// in global memory the selection took 80% of a step at order 128.
template <typename T>
__host__ __device__ inline size_t kog_dyn_ints_end(int nmax, bool gg)        // bytes up to the weights
{
    const size_t g = gg ? 0 : (size_t)(nmax + 1) * nmax * sizeof(T);
    const size_t ints = 2 * (size_t)nmax + 2 * (2 * (size_t)(nmax / 2 + 1) + 2 * (size_t)nmax) + 2 * (size_t)nmax + 8;
    return (g + (2 * kog_piv_elems<T>(nmax) + (size_t)nmax) * sizeof(T) + ints * sizeof(int) + 15) & ~(size_t)15;
}
template <typename T>
__host__ __device__ inline size_t kog_dyn_smem_bytes(int nmax, bool gg, bool wsm)
{
    return kog_dyn_ints_end<T>(nmax, gg) + (wsm ? (size_t)nmax * (nmax - 1) / 2 * sizeof(T) : 0) + 64;
}

// Packed index of the pair i < j: the pairs in lexicographic order (i, j).
__device__ __forceinline__ int dyn_tri(int n, int i, int j) { return i * (2 * n - i - 1) / 2 + (j - i - 1); }

// (w1, k1) ranks before (w2, k2): larger weight, then smaller pair index; k < 0 is no pair.
// The weights are sums of squares (never negative, zero only as +0), so their bit patterns
// order like their values: the comparisons run on the integer pipe, not the FP64 one.
__device__ __forceinline__ uint64_t dyn_key(double w) { return dbits(w); }
__device__ __forceinline__ uint64_t dyn_key(float w) { return fbits(w); }
template <typename T> __device__ __forceinline__ bool dyn_before(T w1, int k1, T w2, int k2)
{
    if (k1 < 0) return false;
    if (k2 < 0) return true;
    const uint64_t a = dyn_key(w1), b = dyn_key(w2);
    return a > b || (a == b && k1 < k2);
}

// Barrier over the nthreads first threads of the block (id 0 with all threads: __syncthreads).
__device__ __forceinline__ void dyn_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

struct dyn_bufs {                      // one step's pairs and groups
    int *pi, *pj, *gi, *gj;
    int *np, *nq;                      // counters in shared memory
};

// Weights of G, the pairs of the next step and their pivot SVDs, by threads t0 = tid <
// tn (the first tn threads of the block, synchronized on barrier `bar`).
template <typename T>
__device__ void dyn_select(const T *G, int ld, int n, T *W, int *used, int *best, dyn_bufs b, T *piv, int ps,
                           int tid, int tn, int bar)
{
    for (int t = tid; t < (n + 1) / 2; t += tn)               // rows t and n-1-t: n-1 pairs a thread
        for (int pass = 0; pass < 2; ++pass) {
            const int i = pass ? n - 1 - t : t;
            if (pass && i == t) break;
            for (int j = i + 1; j < n; ++j) {
                const T gij = G[(size_t)j * ld + i], gji = G[(size_t)i * ld + j];
                W[dyn_tri(n, i, j)] = fma(gji, gji, gij * gij);
            }
        }
    for (int q = tid; q < n; q += tn) { used[q] = 0; best[q] = -2; }
    if (tid == 0) { *b.np = 0; *b.nq = 0; }
    dyn_sync(bar, tn);
    int taken = 0;
    for (;;) {
        for (int i = tid; i < n; i += tn) {
            if (used[i] || (best[i] >= 0 && !used[best[i]])) continue;     // best partner still free
            T bw = T(0); int bk = -1, bj = -1;
            for (int j = 0; j < n; ++j) {
                if (j == i || used[j]) continue;
                const int k = i < j ? dyn_tri(n, i, j) : dyn_tri(n, j, i);
                const T w = W[k];
                if (dyn_before(w, k, bw, bk)) { bw = w; bk = k; bj = j; }
            }
            best[i] = bj;
        }
        dyn_sync(bar, tn);
        for (int i = tid; i < n; i += tn) {
            const int j = best[i];
            if (!used[i] && j > i && best[j] == i) {           // mutually best: taken
                const int a = atomicAdd(b.np, 1);
                b.pi[a] = i; b.pj[a] = j;
                used[i] = 1; used[j] = 1;
            }
        }
        dyn_sync(bar, tn);
        const int now = *b.np;
        if (now == taken) break;                               // no free pair left
        taken = now;
    }
    const int np = taken;
    for (int a = tid; a < np; a += tn) { b.gi[a] = b.pi[a]; b.gj[a] = b.pj[a]; }
    for (int q = tid; q < n; q += tn)
        if (!used[q]) { const int a = np + atomicAdd(b.nq, 1); b.gi[a] = q; b.gj[a] = -1; }
    for (int a = tid; a < np; a += tn) {
        const int i = b.pi[a], j = b.pj[a];
        kog_pivot(G[(size_t)i * ld + i], G[(size_t)i * ld + j], G[(size_t)j * ld + i], G[(size_t)j * ld + j], piv + a, ps);
    }
}

// G <- U-hat^T G V-hat by 2x2 blocks of groups (as kog_rotate_g)
template <typename T>
__device__ __forceinline__ void dyn_rotate_g(T *G, int ld, int n, const dyn_bufs &b, int np, const T *piv, int ps,
                                             int t0, int tn)
{
    const int nq = n - np;
    for (int w2 = t0; w2 < nq * nq; w2 += tn) {
        const int a = w2 % nq, bb = w2 / nq;
        const int ia = b.gi[a], ja = b.gj[a], ib = b.gi[bb], jb = b.gj[bb];
        if (ja < 0 && jb < 0) continue;
        if (a == bb) {
            G[(size_t)ia * ld + ia] = piv[8 * ps + a];
            G[(size_t)ia * ld + ja] = T(0);
            G[(size_t)ja * ld + ia] = T(0);
            G[(size_t)ja * ld + ja] = piv[9 * ps + a];
            continue;
        }
        T *c0 = G + (size_t)ib * ld, *c1 = jb >= 0 ? G + (size_t)jb * ld : nullptr;
        T x00 = c0[ia], x10 = T(0), x01 = T(0), x11 = T(0);
        if (ja >= 0) x10 = c0[ja];
        if (jb >= 0) { x01 = c1[ia]; if (ja >= 0) x11 = c1[ja]; }
        if (ja >= 0) {
            rot2(x00, x10, piv + a, ps);
            if (jb >= 0) rot2(x01, x11, piv + a, ps);
        }
        if (jb >= 0) {
            rot2(x00, x01, piv + 4 * ps + bb, ps);
            if (ja >= 0) rot2(x10, x11, piv + 4 * ps + bb, ps);
        }
        c0[ia] = x00;
        if (ja >= 0) c0[ja] = x10;
        if (jb >= 0) { c1[ia] = x01; if (ja >= 0) c1[ja] = x11; }
    }
}

template <typename T>
__device__ __forceinline__ void dyn_rotate_uv(T *U, T *V, int n, const dyn_bufs &b, int np, const T *piv, int ps,
                                              int t0, int tn)
{
    for (int w2 = t0; w2 < np * n; w2 += tn) {
        const int r = w2 % n, a = w2 / n;
        const int i = b.pi[a], j = b.pj[a];
        rot2(U[(size_t)i * n + r], U[(size_t)j * n + r], piv + a, ps);
        rot2(V[(size_t)i * n + r], V[(size_t)j * n + r], piv + 4 * ps + a, ps);
    }
}

template <typename T, bool GG>
__global__ void __launch_bounds__(512) kog_dynamic(const kog_params<T> P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ kog_sh sh;
    const int nmax = P.nmax, ps = kog_piv_stride(nmax), h = nmax / 2 + 1;
    T *Gs = reinterpret_cast<T *>(smem);
    T *pivb[2];
    pivb[0] = Gs + (GG ? 0 : (size_t)(nmax + 1) * nmax);
    pivb[1] = pivb[0] + kog_piv_elems<T>(nmax);
    T *colsum = pivb[1] + kog_piv_elems<T>(nmax);
    int *perm = reinterpret_cast<int *>(colsum + nmax);
    int *ip = perm + 2 * nmax;
    dyn_bufs bufs[2];
    for (int q = 0; q < 2; ++q) {
        bufs[q].pi = ip; bufs[q].pj = ip + h; bufs[q].gi = ip + 2 * h; bufs[q].gj = ip + 2 * h + nmax;
        ip += 2 * h + 2 * nmax;
    }
    int *used = ip, *best = ip + nmax, *cnt = ip + 2 * nmax;
    bufs[0].np = cnt; bufs[0].nq = cnt + 1; bufs[1].np = cnt + 2; bufs[1].nq = cnt + 3;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (;;) {
        if (tid == 0) sh.slot = atomicAdd(P.queue, 1);
        __syncthreads();
        const int slot = sh.slot;
        __syncthreads();
        if (slot >= P.count) break;
        const kog_desc d = P.desc[slot];
        const int n = d.n, ld = GG ? n : n + 1;
        T *G = GG ? P.gws + d.goff : Gs;
        T *U = P.U + d.off, *V = P.V + d.off, *S = P.S + d.soff;
        T *W = P.wsm ? reinterpret_cast<T *>(smem + kog_dyn_ints_end<T>(nmax, GG))                 // pair weights
                     : P.gws + d.goff + (GG ? (((int64_t)n * n + 1) & ~(int64_t)1) : 0);
        const int k = kog_load(P.A + d.off, G, ld, U, V, n, &sh);
        if (k == INT_MIN) {
            kog_fail(U, V, S, n);
            if (tid == 0) {
                if (P.sweeps) P.sweeps[d.idx] = 0;
                if (P.info) P.info[d.idx] = -1;
            }
            __syncthreads();
            continue;
        }
        T *bc = reinterpret_cast<T *>(&sh.b);
        const T nrm = kog_norm(G, n, ld, false, colsum, bc);
        const T tol = (T(P.tol_factor) * T(n)) * kog_eps<T>::v() * nrm;
        T off = kog_norm(G, n, ld, true, colsum, bc);
        int sw = 0;
        bool go = !(off < tol) && sw < P.max_sweeps && off > T(0);
        // the selecting warps: enough for one thread per index, at most half the block
        const int nw = (nt + 31) >> 5;
        int w0 = (n + 31) >> 5;
        if (w0 > nw / 2) w0 = nw / 2;
        const bool split = w0 >= 1 && nt - 32 * w0 >= 32;
        int cur = 0;
        if (go) {
            dyn_select(G, ld, n, W, used, best, bufs[0], pivb[0], ps, tid, nt, 0);
            __syncthreads();
        }
        while (go) {
            for (int st = 0; st < n; ++st) {
                const int nxt = cur ^ 1;
                const int np = *bufs[cur].np;
                dyn_rotate_g(G, ld, n, bufs[cur], np, pivb[cur], ps, tid, nt);       // G_{k+1}
                __syncthreads();
                // the pairs of the next step (the first of the next sweep after the last
                // one: unused when the sweeps end) beside the U and V updates of this one
                if (split) {
                    if (tid < 32 * w0) dyn_select(G, ld, n, W, used, best, bufs[nxt], pivb[nxt], ps, tid, 32 * w0, 1);
                    else dyn_rotate_uv(U, V, n, bufs[cur], np, pivb[cur], ps, tid - 32 * w0, nt - 32 * w0);
                } else {
                    dyn_rotate_uv(U, V, n, bufs[cur], np, pivb[cur], ps, tid, nt);
                    __syncthreads();
                    dyn_select(G, ld, n, W, used, best, bufs[nxt], pivb[nxt], ps, tid, nt, 0);
                }
                __syncthreads();
                cur = nxt;
            }
            ++sw;
            off = kog_norm(G, n, ld, true, colsum, bc);
            go = !(off < tol) && sw < P.max_sweeps && off > T(0);
        }
        kog_finish(G, ld, U, V, S, n, k, colsum, perm, G);
        if (tid == 0) {
            if (P.sweeps) P.sweeps[d.idx] = sw;
            if (P.info) P.info[d.idx] = (off < tol || off == T(0)) ? 0 : 1;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// per-step form: state per matrix in the workspace
// ---------------------------------------------------------------------------------------
template <typename T> struct kog_state {
    T tol, off;
    int k, sw, active, bad;
};

template <typename T>
__global__ void __launch_bounds__(256) kogp_init(const kog_params<T> P, kog_state<T> *state)
{
    __shared__ kog_sh sh;
    extern __shared__ __align__(16) unsigned char smem[];
    T *colsum = reinterpret_cast<T *>(smem);
    const kog_desc d = P.desc[blockIdx.x];
    const int n = d.n;
    T *G = P.gws + d.goff, *U = P.U + d.off, *V = P.V + d.off;
    const int k = kog_load(P.A + d.off, G, n, U, V, n, &sh);
    kog_state<T> &s = state[blockIdx.x];
    if (k == INT_MIN) {
        kog_fail(U, V, P.S + d.soff, n);
        if (threadIdx.x == 0) { s.bad = 1; s.active = 0; s.sw = 0; s.k = 0; }
        return;
    }
    T *bc = reinterpret_cast<T *>(&sh.b);
    const T nrm = kog_norm(G, n, n, false, colsum, bc);
    const T tol = (T(P.tol_factor) * T(n)) * kog_eps<T>::v() * nrm;
    const T off = kog_norm(G, n, n, true, colsum, bc);
    if (threadIdx.x == 0) {
        s.tol = tol; s.off = off; s.k = k; s.sw = 0; s.bad = 0;
        s.active = (!(off < tol) && P.max_sweeps > 0 && off > T(0)) ? 1 : 0;
        if (s.active) atomicAdd(P.queue, 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(128) kogp_pivots(const kog_params<T> P, const kog_state<T> *state, T *pivws,
                                                   const int64_t *pivoff, int st)
{
    const int m = blockIdx.y;
    if (!state[m].active) return;
    const kog_desc d = P.desc[m];
    if (st >= d.n) return;
    const int np = modulus_count(d.n, st);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const T *G = P.gws + d.goff;
    const int n = d.n;
    int i, j;
    modulus_pair(n, st, p, i, j);
    kog_pivot(G[(size_t)i * n + i], G[(size_t)i * n + j], G[(size_t)j * n + i], G[(size_t)j * n + j],
              pivws + pivoff[m] + 10 * p);
}

template <typename T>
__global__ void __launch_bounds__(256) kogp_rows(const kog_params<T> P, const kog_state<T> *state, const T *pivws,
                                                 const int64_t *pivoff, int st)
{
    const int m = blockIdx.y;
    if (!state[m].active) return;
    const kog_desc d = P.desc[m];
    const int n = d.n;
    if (st >= n) return;
    const int np = modulus_count(n, st);
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= np * n) return;
    const int p = w % np, c = w / np;
    int i, j;
    modulus_pair(n, st, p, i, j);
    T *G = P.gws + d.goff;
    rot2(G[(size_t)c * n + i], G[(size_t)c * n + j], pivws + pivoff[m] + 10 * p);
}

template <typename T>
__global__ void __launch_bounds__(256) kogp_cols(const kog_params<T> P, const kog_state<T> *state, const T *pivws,
                                                 const int64_t *pivoff, int st)
{
    const int m = blockIdx.y;
    if (!state[m].active) return;
    const kog_desc d = P.desc[m];
    const int n = d.n;
    if (st >= n) return;
    const int np = modulus_count(n, st);
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= np * n) return;
    const int r = w % n, p = w / n;
    int i, j;
    modulus_pair(n, st, p, i, j);
    T *G = P.gws + d.goff, *U = P.U + d.off, *V = P.V + d.off;
    const T *mm = pivws + pivoff[m] + 10 * p;
    if (r == i || r == j) {
        G[(size_t)i * n + r] = (r == i) ? mm[8] : T(0);
        G[(size_t)j * n + r] = (r == j) ? mm[9] : T(0);
    } else {
        rot2(G[(size_t)i * n + r], G[(size_t)j * n + r], mm + 4);
    }
    rot2(U[(size_t)i * n + r], U[(size_t)j * n + r], mm);
    rot2(V[(size_t)i * n + r], V[(size_t)j * n + r], mm + 4);
}

template <typename T>
__global__ void __launch_bounds__(256) kogp_offnorm(const kog_params<T> P, kog_state<T> *state)
{
    __shared__ kog_sh sh;
    extern __shared__ __align__(16) unsigned char smem[];
    T *colsum = reinterpret_cast<T *>(smem);
    kog_state<T> &s = state[blockIdx.x];
    if (!s.active) return;
    const kog_desc d = P.desc[blockIdx.x];
    T *bc = reinterpret_cast<T *>(&sh.b);
    const T off = kog_norm(P.gws + d.goff, d.n, d.n, true, colsum, bc);
    if (threadIdx.x == 0) {
        s.off = off;
        s.sw += 1;
        s.active = (!(off < s.tol) && s.sw < P.max_sweeps && off > T(0)) ? 1 : 0;
        if (s.active) atomicAdd(P.queue, 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) kogp_finish(const kog_params<T> P, const kog_state<T> *state)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const kog_state<T> s = state[blockIdx.x];
    if (s.bad) {
        if (threadIdx.x == 0) {
            const kog_desc d = P.desc[blockIdx.x];
            if (P.sweeps) P.sweeps[d.idx] = 0;
            if (P.info) P.info[d.idx] = -1;
        }
        return;
    }
    const kog_desc d = P.desc[blockIdx.x];
    const int n = d.n;
    T *dg = reinterpret_cast<T *>(smem);
    int *perm = reinterpret_cast<int *>(dg + P.nmax);
    T *G = P.gws + d.goff;
    kog_finish(G, n, P.U + d.off, P.V + d.off, P.S + d.soff, n, s.k, dg, perm, G);
    if (threadIdx.x == 0) {
        if (P.sweeps) P.sweeps[d.idx] = s.sw;
        if (P.info) P.info[d.idx] = (s.off < s.tol || s.off == T(0)) ? 0 : 1;
    }
}

// ---------------------------------------------------------------------------------------
// sigma gradient: dA = U diag(dS) V^T, one block per (column tile, matrix)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) kog_sigma_bwd_kernel(const kog_desc *desc, const T *U, const T *V, const T *dS,
                                                            T *dA)
{
    const kog_desc d = desc[blockIdx.y];
    const int n = d.n;
    const T *u = U + d.off, *v = V + d.off, *ds = dS + d.soff;
    T *a = dA + d.off;
    const int nn = n * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
        const int r = e % n, c = e / n;
        T acc = T(0);
        for (int q = 0; q < n; ++q) acc = fma(u[(size_t)q * n + r] * ds[q], v[(size_t)q * n + c], acc);
        a[e] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// host side: plan, workspace layout, autotuner, graph cache
// ---------------------------------------------------------------------------------------
template <typename T> struct kog_limits;
template <> struct kog_limits<double> { static constexpr int SMEM_MAX_N = 128; };
template <> struct kog_limits<float> { static constexpr int SMEM_MAX_N = 224; };

// Order buckets, one persistent launch each: orders up to 32, 48, ..., 128 (G in shared
// memory), up to the shared-memory limit, and the rest (G in the workspace).  A bucket's
// shared memory is sized by its largest order, so narrow buckets let several CTAs share an
// SM where G is small: while one matrix waits on the serial 2x2 SVDs of its next step,
// another's rotations use the FP64 pipe.
static constexpr int BUCKET_TOP[] = {32, 48, 64, 80, 96, 112, 128};
static constexpr int NFIXED = 7;
static constexpr int NBUCKETS = NFIXED + 2;
static constexpr int BUCKET_GLOBAL = NBUCKETS - 1;
// the work counters of the buckets, QUEUE_STRIDE ints apart in the first 512 bytes of the scratch
static constexpr int QUEUE_STRIDE = 8;
static_assert(NBUCKETS * QUEUE_STRIDE <= 128, "bucket work counters exceed their 512 bytes");

static int bucket_of(int n, int smem_max)
{
    if (n <= smem_max)
        for (int b = 0; b < NFIXED; ++b)
            if (n <= BUCKET_TOP[b]) return b;
    return n <= smem_max ? NFIXED : BUCKET_GLOBAL;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T> struct kog_plan {
    std::vector<kog_desc> desc;                      // sorted: bucket, then decreasing n
    int bstart[NBUCKETS + 1];
    int bnmax[NBUCKETS];
    size_t off_desc, off_queue, off_g, off_state, off_piv, off_pivoff, total;
    std::vector<int64_t> pivoff;                     // per-step form
    bool plain, dyn;
};

template <typename T>
static int make_plan(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, int32_t flags,
                     kog_plan<T> &pl)
{
    const int smax = kog_limits<T>::SMEM_MAX_N;
    pl.plain = (flags & K2SVD_KOG_PLAIN) != 0;
    pl.dyn = (flags & K2SVD_KOG_DYNAMIC) != 0;
    pl.desc.resize((size_t)batch);
    for (int64_t i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 4096) return -2;
        kog_desc &d = pl.desc[(size_t)i];
        d.n = n[i]; d.idx = (int32_t)i; d.off = offs ? offs[i] : 0; d.soff = soffs ? soffs[i] : 0; d.goff = 0;
    }
    std::stable_sort(pl.desc.begin(), pl.desc.end(), [&](const kog_desc &a, const kog_desc &b) {
        int ba = bucket_of(a.n, smax), bb = bucket_of(b.n, smax);
        if (ba != bb) return ba < bb;
        return a.n > b.n;
    });
    for (int b = 0; b <= NBUCKETS; ++b) pl.bstart[b] = 0;
    for (int b = 0; b < NBUCKETS; ++b) pl.bnmax[b] = 0;
    for (size_t i = 0; i < pl.desc.size(); ++i) {
        int b = bucket_of(pl.desc[i].n, smax);
        pl.bstart[b + 1] = (int)i + 1;
        pl.bnmax[b] = std::max(pl.bnmax[b], pl.desc[i].n);
    }
    for (int b = 1; b <= NBUCKETS; ++b) pl.bstart[b] = std::max(pl.bstart[b], pl.bstart[b - 1]);
    // scratch: G for every matrix in the per-step form and for the global bucket in the
    // persistent form, then the n(n-1)/2 pair weights of every matrix with the dynamic ordering
    int64_t g = 0;
    for (auto &d : pl.desc) {
        const bool gg = pl.plain || bucket_of(d.n, smax) == BUCKET_GLOBAL;
        if (gg || pl.dyn) {
            d.goff = g;
            if (gg) g += ((int64_t)d.n * d.n + 1) & ~(int64_t)1;
            if (pl.dyn) g += ((int64_t)d.n * (d.n - 1) / 2 + 1) & ~(int64_t)1;
        }
    }
    size_t off = 0;
    pl.off_queue = off; off = align256(off + 128 * sizeof(int));
    pl.off_desc = off; off = align256(off + pl.desc.size() * sizeof(kog_desc));
    pl.off_g = off; off = align256(off + (size_t)g * sizeof(T));
    pl.off_state = off;
    pl.off_piv = off;
    pl.off_pivoff = off;
    if (pl.plain) {
        off = align256(off + pl.desc.size() * sizeof(kog_state<T>));
        pl.pivoff.resize(pl.desc.size());
        int64_t pv = 0;
        for (size_t i = 0; i < pl.desc.size(); ++i) { pl.pivoff[i] = pv; pv += (int64_t)(pl.desc[i].n / 2 + 1) * 10; }
        pl.off_pivoff = off; off = align256(off + pl.desc.size() * sizeof(int64_t));
        pl.off_piv = off; off = align256(off + (size_t)pv * sizeof(T));
    }
    pl.total = off;
    return 0;
}

struct tune_key {
    int dev, tsize, bucket, dyn;
    bool operator<(const tune_key &o) const
    {
        return std::tie(dev, tsize, bucket, dyn) < std::tie(o.dev, o.tsize, o.bucket, o.dyn);
    }
};
static std::mutex g_mu;
static std::map<tune_key, int> g_tuned;

static int default_threads(int nmax) { return nmax <= 32 ? 64 : (nmax <= 64 ? 256 : 512); }

template <typename T, bool GG, bool DYN>
static cudaError_t launch_bucket_k(const kog_params<T> &Pin, int threads, cudaStream_t st, int *queue_dev, int prio)
{
    kog_params<T> P = Pin;
    const bool uvs = !GG && !DYN && P.nmax <= KOG_UVS_MAX;
    auto kern = DYN ? kog_dynamic<T, GG>
                    : (P.nmax <= 64 ? (uvs ? kog_persistent<T, GG, 2, true> : kog_persistent<T, GG, 2, false>)
                       : threads > 512 ? kog_persistent<T, GG, 1, false, 1024> : kog_persistent<T, GG, 1, false>);
    size_t smem = kog_smem_bytes<T>(P.nmax, GG, uvs);
    P.wsm = 0;
    if (DYN) {                                         // the weights in shared memory when they fit
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return cudaErrorUnknown;
        P.wsm = (!GG && kog_dyn_smem_bytes<T>(P.nmax, GG, true) <= (size_t)optin) ? 1 : 0;
        smem = kog_dyn_smem_bytes<T>(P.nmax, GG, P.wsm != 0);
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = 0;
    if (grid_for(kern, threads, smem, &blocks) != 0) return cudaErrorUnknown;
    if (blocks > P.count) blocks = P.count;
    if (blocks < 1) return cudaSuccess;
    e = cudaMemsetAsync(queue_dev, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = prio != 0 ? 1 : 0;                 // else the stream's own priority
    return cudaLaunchKernelEx(&cfg, kern, P);
}

template <typename T>
static cudaError_t launch_bucket(const kog_params<T> &P, int bucket, bool dyn, int threads, cudaStream_t st, int *queue_dev,
                                 int prio = 0)
{
    if (bucket == BUCKET_GLOBAL)
        return dyn ? launch_bucket_k<T, true, true>(P, threads, st, queue_dev, prio) : launch_bucket_k<T, true, false>(P, threads, st, queue_dev, prio);
    return dyn ? launch_bucket_k<T, false, true>(P, threads, st, queue_dev, prio) : launch_bucket_k<T, false, false>(P, threads, st, queue_dev, prio);
}

// Streams and events of the concurrent bucket launches, per device (created on first use,
// kept until exit).  g_fork_mu serialises their use by concurrent callers; a graph capture
// holds it until the capture ends, since the streams belong to the capture until then.
struct kog_fork {
    cudaStream_t aux[NBUCKETS];
    cudaEvent_t fork, join[NBUCKETS];
    int least, greatest;
};
static std::recursive_mutex g_fork_mu;
static std::map<int, kog_fork> g_forks;

static kog_fork *get_fork(int dev)
{
    auto it = g_forks.find(dev);
    if (it != g_forks.end()) return &it->second;
    kog_fork f;
    if (cudaDeviceGetStreamPriorityRange(&f.least, &f.greatest) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    for (int b = 0; b < NBUCKETS; ++b) {
        const int pr = f.least - (b * (f.least - f.greatest)) / (NBUCKETS - 1);
        if (cudaStreamCreateWithPriority(&f.aux[b], cudaStreamNonBlocking, pr) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&f.join[b], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    return &(g_forks[dev] = f);
}

// With fork, the buckets run concurrently, each on a stream of its own, largest orders at
// the highest priority: their CTAs are placed first, and the CTAs of the smaller orders take
// the SMs that the larger buckets leave, so no bucket's tail leaves SMs idle.
template <typename T>
static cudaError_t launch_persistent(const kog_plan<T> &pl, kog_params<T> base, const int *threads, cudaStream_t st,
                                     unsigned char *ws, bool fork = false)
{
    const kog_desc *ddesc = reinterpret_cast<const kog_desc *>(ws + pl.off_desc);
    int *queues = reinterpret_cast<int *>(ws + pl.off_queue);
    int used = 0;
    for (int b = 0; b < NBUCKETS; ++b) used += pl.bstart[b + 1] > pl.bstart[b];
    if (fork && used > 1) {
        int dev;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
        std::lock_guard<std::recursive_mutex> lk(g_fork_mu);
        kog_fork *f = get_fork(dev);
        if (!f) return cudaErrorUnknown;
        cudaError_t e = cudaEventRecord(f->fork, st);
        if (e != cudaSuccess) return e;
        for (int b = NBUCKETS - 1; b >= 0; --b) {
            int cnt = pl.bstart[b + 1] - pl.bstart[b];
            if (cnt <= 0) continue;
            kog_params<T> P = base;
            P.desc = ddesc + pl.bstart[b];
            P.count = cnt;
            P.queue = queues + QUEUE_STRIDE * b;
            P.nmax = pl.bnmax[b];
            const int pr = f->least - (b * (f->least - f->greatest)) / (NBUCKETS - 1);
            if ((e = cudaStreamWaitEvent(f->aux[b], f->fork, 0)) != cudaSuccess) return e;
            if ((e = launch_bucket<T>(P, b, pl.dyn, threads[b], f->aux[b], P.queue, pr)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(f->join[b], f->aux[b])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, f->join[b], 0)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int b = 0; b < NBUCKETS; ++b) {
        int cnt = pl.bstart[b + 1] - pl.bstart[b];
        if (cnt <= 0) continue;
        kog_params<T> P = base;
        P.desc = ddesc + pl.bstart[b];
        P.count = cnt;
        P.queue = queues + QUEUE_STRIDE * b;
        P.nmax = pl.bnmax[b];
        cudaError_t e = launch_bucket<T>(P, b, pl.dyn, threads[b], st, P.queue);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Pick the block size of each bucket by timing a sample (the largest matrices of the
// bucket, four per SM, so that a block size that fits several CTAs on an SM can show it)
// on the caller's arrays; results are launch-shape independent.
template <typename T>
static int autotune(const kog_plan<T> &pl, const kog_params<T> &base, cudaStream_t st, unsigned char *ws, int dev,
                    int *threads, bool tune)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int b = 0; b < NBUCKETS; ++b) {
        int cnt = pl.bstart[b + 1] - pl.bstart[b];
        threads[b] = default_threads(pl.bnmax[b]);
        if (cnt <= 0) continue;
        tune_key key{dev, (int)sizeof(T), b, pl.dyn ? 1 : 0};
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) { threads[b] = it->second; continue; }
        }
        if (!tune) continue;
        const int cand[6] = {32, 64, 128, 256, 512, 1024};
        kog_params<T> P = base;
        P.desc = reinterpret_cast<const kog_desc *>(ws + pl.off_desc) + pl.bstart[b];
        P.count = std::min(cnt, 4 * sms);
        P.queue = reinterpret_cast<int *>(ws + pl.off_queue) + QUEUE_STRIDE * b;
        P.nmax = pl.bnmax[b];
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return K2SVD_ECUDA;
        float best = 1e30f;
        int bestt = threads[b];
        for (int t : cand) {
            if (t > 512 && (pl.dyn || P.nmax <= 64)) continue;   // 1024 threads: the 64-register kernel of orders > 64
            cudaEventRecord(e0, st);
            cudaError_t e = launch_bucket<T>(P, b, pl.dyn, t, st, P.queue);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0); cudaEventDestroy(e1);
                return K2SVD_ECUDA;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bestt = t; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        threads[b] = bestt;
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[key] = bestt;
    }
    return 0;
}

// Cache of instantiated graphs for repeated calls with the same arguments.
struct graph_key {
    std::vector<int64_t> sig;
    bool operator<(const graph_key &o) const { return sig < o.sig; }
};
static std::map<graph_key, cudaGraphExec_t> g_graphs;

template <typename T>
static int kogbet_plain(const kog_plan<T> &pl, kog_params<T> base, cudaStream_t st, unsigned char *ws)
{
    const int m = (int)pl.desc.size();
    kog_desc *ddesc = reinterpret_cast<kog_desc *>(ws + pl.off_desc);
    kog_state<T> *state = reinterpret_cast<kog_state<T> *>(ws + pl.off_state);
    T *pivws = reinterpret_cast<T *>(ws + pl.off_piv);
    int64_t *pivoff = reinterpret_cast<int64_t *>(ws + pl.off_pivoff);
    int *counter = reinterpret_cast<int *>(ws + pl.off_queue);
    if (cudaMemcpyAsync(pivoff, pl.pivoff.data(), pl.pivoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return K2SVD_ECUDA;
    int nmax = 0;
    for (auto &d : pl.desc) nmax = std::max(nmax, d.n);
    kog_params<T> P = base;
    P.desc = ddesc; P.count = m; P.queue = counter; P.nmax = nmax;
    const size_t sm_norm = (size_t)nmax * sizeof(T) + 2 * (size_t)nmax * sizeof(int) + 64;
    if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return K2SVD_ECUDA;
    kogp_init<T><<<m, 256, sm_norm, st>>>(P, state);
    int remaining = 0;
    if (cudaMemcpyAsync(&remaining, counter, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return K2SVD_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return K2SVD_ECUDA;
    const int maxpairs = nmax / 2 + 1, maxitems = maxpairs * nmax;
    for (int sw = 0; sw < base.max_sweeps && remaining > 0; ++sw) {
        for (int s = 0; s < nmax; ++s) {
            kogp_pivots<T><<<dim3((maxpairs + 127) / 128, m), 128, 0, st>>>(P, state, pivws, pivoff, s);
            kogp_rows<T><<<dim3((maxitems + 255) / 256, m), 256, 0, st>>>(P, state, pivws, pivoff, s);
            kogp_cols<T><<<dim3((maxitems + 255) / 256, m), 256, 0, st>>>(P, state, pivws, pivoff, s);
        }
        if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return K2SVD_ECUDA;
        kogp_offnorm<T><<<m, 256, sm_norm, st>>>(P, state);
        if (cudaMemcpyAsync(&remaining, counter, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return K2SVD_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return K2SVD_ECUDA;
    }
    kogp_finish<T><<<m, 256, sm_norm, st>>>(P, state);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

template <typename T>
static int kogbet_ws(int64_t batch, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    if (batch < 0) return -1;
    if (batch > 0 && !n) return -2;
    if (!ws_bytes) return -4;
    kog_plan<T> pl;
    int rc = make_plan<T>(batch, n, nullptr, nullptr, flags, pl);
    if (rc) return rc;
    *ws_bytes = pl.total;
    return 0;
}

template <typename T>
static int kogbet(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const T *A, T *U, T *V,
                  T *S, int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor, int32_t flags,
                  void *workspace, size_t ws_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (batch == 0) return 0;
    if (!n) return -2;
    if (!offs) return -3;
    if (!soffs) return -4;
    if (!A) return -5;
    if (!U) return -6;
    if (!V) return -7;
    if (!S) return -8;
    if (max_sweeps < 0) return -11;
    if (!(tol_factor > 0)) return -12;
    if (flags & ~(K2SVD_KOG_PLAIN | K2SVD_KOG_GRAPH | K2SVD_KOG_NOTUNE | K2SVD_KOG_DYNAMIC)) return -13;
    if ((flags & K2SVD_KOG_PLAIN) && (flags & (K2SVD_KOG_GRAPH | K2SVD_KOG_DYNAMIC))) return -13;
    if (!workspace || ((uintptr_t)workspace & 255)) return -14;
    kog_plan<T> pl;
    int rc = make_plan<T>(batch, n, offs, soffs, flags, pl);
    if (rc) return rc;
    if (ws_bytes < pl.total) return -15;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = capture_guard(st)) != 0) return rc;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    if (cudaMemcpyAsync(ws + pl.off_desc, pl.desc.data(), pl.desc.size() * sizeof(kog_desc), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return K2SVD_ECUDA;
    kog_params<T> base;
    base.desc = nullptr; base.count = 0; base.queue = nullptr;
    base.A = A; base.U = U; base.V = V; base.S = S; base.sweeps = sweeps; base.info = info;
    base.gws = reinterpret_cast<T *>(ws + pl.off_g);
    base.max_sweeps = max_sweeps; base.tol_factor = tol_factor; base.nmax = 0; base.wsm = 0;
    if (pl.plain) {
        if (batch > 65535) return -1;                  // one grid row per matrix
        return kogbet_plain<T>(pl, base, st, ws);
    }
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    int threads[NBUCKETS];
    const char *env = getenv("K2SVD_TUNE");
    bool tune = !(flags & K2SVD_KOG_NOTUNE) && !(env && env[0] == '0');
    if (autotune<T>(pl, base, st, ws, dev, threads, tune) != 0) return K2SVD_ECUDA;
    if (!(flags & K2SVD_KOG_GRAPH))
        return launch_persistent<T>(pl, base, threads, st, ws, true) == cudaSuccess ? 0 : K2SVD_ECUDA;
    // graph: cached per (device, type, arguments, plan shape, block sizes)
    graph_key key;
    key.sig = {dev, (int64_t)sizeof(T), batch, (int64_t)(uintptr_t)A, (int64_t)(uintptr_t)U, (int64_t)(uintptr_t)V,
               (int64_t)(uintptr_t)S, (int64_t)(uintptr_t)sweeps, (int64_t)(uintptr_t)info, max_sweeps,
               (int64_t)(uintptr_t)workspace, flags};
    int64_t tbits;
    std::memcpy(&tbits, &tol_factor, sizeof tbits);
    key.sig.push_back(tbits);
    for (int b = 0; b < NBUCKETS; ++b) { key.sig.push_back(threads[b]); key.sig.push_back(pl.bstart[b + 1]); key.sig.push_back(pl.bnmax[b]); }
    for (auto &d : pl.desc) { key.sig.push_back(d.n); key.sig.push_back(d.off); key.sig.push_back(d.soff); }
    {
        // a cached graph is launched under the cache's lock, so no other caller can evict
        // and destroy it in between
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) return cudaGraphLaunch(it->second, st) == cudaSuccess ? 0 : K2SVD_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    {
        // the bucket streams join this capture until it ends: no other caller may enqueue
        // on them meanwhile (the lock is the one launch_persistent takes, held throughout)
        std::lock_guard<std::recursive_mutex> fk(g_fork_mu);
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return K2SVD_ECUDA;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { cudaStreamDestroy(cap); return K2SVD_ECUDA; }
        cudaError_t e = launch_persistent<T>(pl, base, threads, cap, ws, true);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || e2 != cudaSuccess) return K2SVD_ECUDA;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return K2SVD_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_graphs.find(key);
    if (it != g_graphs.end()) {                      // another caller cached the same graph
        cudaGraphExecDestroy(exec);
        exec = it->second;
    } else {
        if (g_graphs.size() >= 16) {                 // bounded cache
            cudaGraphExecDestroy(g_graphs.begin()->second);
            g_graphs.erase(g_graphs.begin());
        }
        g_graphs[key] = exec;
    }
    return cudaGraphLaunch(exec, st) == cudaSuccess ? 0 : K2SVD_ECUDA;
}

template <typename T>
static int kog_sigma_bwd(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const T *U,
                         const T *V, const T *dS, T *dA, void *workspace, size_t ws_bytes, void *stream)
{
    if (batch < 0 || batch > 65535) return -1;
    if (batch == 0) return 0;
    if (!n) return -2;
    if (!offs) return -3;
    if (!soffs) return -4;
    if (!U) return -5;
    if (!V) return -6;
    if (!dS) return -7;
    if (!dA) return -8;
    if (!workspace || ((uintptr_t)workspace & 255)) return -9;
    if (ws_bytes < (size_t)batch * sizeof(kog_desc)) return -10;
    std::vector<kog_desc> desc((size_t)batch);
    int nmax = 1;
    for (int64_t i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 4096) return -2;
        desc[(size_t)i] = kog_desc{n[i], (int32_t)i, offs[i], soffs[i], 0};
        nmax = std::max(nmax, (int)n[i]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = capture_guard(st)) return rc;
    kog_desc *d_desc = static_cast<kog_desc *>(workspace);
    if (cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(kog_desc), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return K2SVD_ECUDA;
    int xb = std::min(64, (nmax * nmax + 255) / 256);
    kog_sigma_bwd_kernel<T><<<dim3(xb, (unsigned)batch), 256, 0, st>>>(d_desc, U, V, dS, dA);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : K2SVD_ECUDA;
}

// ---------------------------------------------------------------------------------------
// Allocation-free entry (k2svd_dkogbet_noalloc): the same persistent launches with the
// scratch in a fixed array of every device that loads this library.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_kog_scratch[K2SVD_KOG_NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEV = 64;
static std::mutex g_scratch_mu;
static void *g_scratch_ptr[NOALLOC_MAX_DEV];
// host staging of the descriptor table: static storage, so the call allocates nothing
static kog_desc g_noalloc_desc[K2SVD_KOG_NOALLOC_BYTES / sizeof(kog_desc)];

// Address of this device's scratch array, looked up once per device with it current.
static int noalloc_scratch(void **p)
{
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEV) return K2SVD_ECUDA;
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_kog_scratch) != cudaSuccess || !ptr) return K2SVD_ECUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *p = g_scratch_ptr[dev];
    return 0;
}

static int kogbet_noalloc(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const double *A,
                          double *U, double *V, double *S, int32_t *sweeps, int32_t *info, int32_t max_sweeps,
                          double tol_factor, void *stream)
{
    if (batch < 0) return -1;
    if (batch == 0) return 0;
    if (!n) return -2;
    if (!offs) return -3;
    if (!soffs) return -4;
    if (!A) return -5;
    if (!U) return -6;
    if (!V) return -7;
    if (!S) return -8;
    if (max_sweeps < 0) return -11;
    if (!(tol_factor > 0)) return -12;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = capture_guard(st)) return rc;
    const int smax = kog_limits<double>::SMEM_MAX_N;
    // scratch layout as the workspace of the persistent form: queues, descriptors, G of orders > 128
    size_t bytes = align256(128 * sizeof(int)) + align256((size_t)batch * sizeof(kog_desc));
    int64_t g = 0;
    for (int64_t i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 4096) return -2;
        if (bucket_of(n[i], smax) == BUCKET_GLOBAL) g += ((int64_t)n[i] * n[i] + 1) & ~(int64_t)1;
    }
    bytes += align256((size_t)g * sizeof(double));
    if (bytes > (size_t)K2SVD_KOG_NOALLOC_BYTES) return K2SVD_ENOSPACE;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != 0) return K2SVD_ECUDA;
    kog_desc *desc = g_noalloc_desc;
    for (int64_t i = 0; i < batch; ++i) desc[i] = kog_desc{n[i], (int32_t)i, offs[i], soffs[i], 0};
    // bucket, then decreasing order, then index: the order of the persistent form's plan
    std::sort(desc, desc + batch, [&](const kog_desc &a, const kog_desc &b) {
        int ba = bucket_of(a.n, smax), bb = bucket_of(b.n, smax);
        if (ba != bb) return ba < bb;
        if (a.n != b.n) return a.n > b.n;
        return a.idx < b.idx;
    });
    kog_plan<double> pl;                              // shape only; no containers are filled
    for (int b = 0; b <= NBUCKETS; ++b) pl.bstart[b] = 0;
    for (int b = 0; b < NBUCKETS; ++b) pl.bnmax[b] = 0;
    int64_t goff = 0;
    for (int64_t i = 0; i < batch; ++i) {
        int b = bucket_of(desc[i].n, smax);
        pl.bstart[b + 1] = (int)i + 1;
        pl.bnmax[b] = std::max(pl.bnmax[b], desc[i].n);
        if (b == BUCKET_GLOBAL) { desc[i].goff = goff; goff += ((int64_t)desc[i].n * desc[i].n + 1) & ~(int64_t)1; }
    }
    for (int b = 1; b <= NBUCKETS; ++b) pl.bstart[b] = std::max(pl.bstart[b], pl.bstart[b - 1]);
    pl.off_queue = 0;
    pl.off_desc = align256(128 * sizeof(int));
    pl.off_g = pl.off_desc + align256((size_t)batch * sizeof(kog_desc));
    pl.plain = false;
    pl.dyn = false;
    unsigned char *ws = static_cast<unsigned char *>(scratch);
    if (cudaMemcpyAsync(ws + pl.off_desc, desc, (size_t)batch * sizeof(kog_desc), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return K2SVD_ECUDA;
    kog_params<double> base;
    base.desc = nullptr; base.count = 0; base.queue = nullptr;
    base.A = A; base.U = U; base.V = V; base.S = S; base.sweeps = sweeps; base.info = info;
    base.gws = reinterpret_cast<double *>(ws + pl.off_g);
    base.max_sweeps = max_sweeps; base.tol_factor = tol_factor; base.nmax = 0; base.wsm = 0;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return K2SVD_ECUDA;
    int threads[NBUCKETS];
    for (int b = 0; b < NBUCKETS; ++b) {             // tuned block sizes if known, else defaults
        threads[b] = default_threads(pl.bnmax[b]);
        std::lock_guard<std::mutex> lk2(g_mu);
        auto it = g_tuned.find(tune_key{dev, (int)sizeof(double), b, 0});
        if (it != g_tuned.end()) threads[b] = it->second;
    }
    return launch_persistent<double>(pl, base, threads, st, ws) == cudaSuccess ? 0 : K2SVD_ECUDA;
}

}  // namespace k2

extern "C" {

int k2svd_dkogbet_noalloc(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const double *A,
                          double *U, double *V, double *S, int32_t *sweeps, int32_t *info, int32_t max_sweeps,
                          double tol_factor, void *stream)
{
    return k2::kogbet_noalloc(batch, n, offs, soffs, A, U, V, S, sweeps, info, max_sweeps, tol_factor, stream);
}

int k2svd_dkogbet_ws(int64_t batch, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    return k2::kogbet_ws<double>(batch, n, flags, ws_bytes);
}
int k2svd_skogbet_ws(int64_t batch, const int32_t *n, int32_t flags, size_t *ws_bytes)
{
    return k2::kogbet_ws<float>(batch, n, flags, ws_bytes);
}
int k2svd_dkogbet(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const double *A, double *U,
                  double *V, double *S, int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor,
                  int32_t flags, void *workspace, size_t ws_bytes, void *stream)
{
    return k2::kogbet<double>(batch, n, offs, soffs, A, U, V, S, sweeps, info, max_sweeps, tol_factor, flags, workspace,
                              ws_bytes, stream);
}
int k2svd_skogbet(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const float *A, float *U,
                  float *V, float *S, int32_t *sweeps, int32_t *info, int32_t max_sweeps, double tol_factor,
                  int32_t flags, void *workspace, size_t ws_bytes, void *stream)
{
    return k2::kogbet<float>(batch, n, offs, soffs, A, U, V, S, sweeps, info, max_sweeps, tol_factor, flags, workspace,
                             ws_bytes, stream);
}
int k2svd_dkog_sigma_bwd(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const double *U,
                         const double *V, const double *dS, double *dA, void *workspace, size_t ws_bytes, void *stream)
{
    return k2::kog_sigma_bwd<double>(batch, n, offs, soffs, U, V, dS, dA, workspace, ws_bytes, stream);
}
int k2svd_skog_sigma_bwd(int64_t batch, const int32_t *n, const int64_t *offs, const int64_t *soffs, const float *U,
                         const float *V, const float *dS, float *dA, void *workspace, size_t ws_bytes, void *stream)
{
    return k2::kog_sigma_bwd<float>(batch, n, offs, soffs, U, V, dS, dA, workspace, ws_bytes, stream);
}

}  // extern "C"
