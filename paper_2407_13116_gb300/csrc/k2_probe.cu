// Pipe-throughput probes (include/k2probe.h): the roofline denominators of the 2x2 SVD
// kernels, measured on the device at hand.
#include <cstdint>
#include <cuda_runtime.h>

#include "k2probe.h"
#include "k2_fp.cuh"

namespace {

constexpr int CHAINS = 8;

template <typename T, int OP>
__global__ void probe_kernel(T *out, int iters, T seed)
{
    T x[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x[i] = seed + T(threadIdx.x) * T(1e-7) + T(i) * T(1e-3);
    const T y = T(1.0000001), z = T(1e-9);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) {
            if (OP == 0) x[i] = fma(x[i], y, z);
            else if (OP == 1) x[i] = x[i] / (y + T(i));
            else x[i] = sqrt(x[i] + z);
        }
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int OP>
int run(double *rate)
{
    int dev, sms;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1000;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1000;
    const int threads = 256, blocks = sms * 8;
    const int iters = (OP == 0) ? 4096 : 512;
    T *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1000;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        probe_kernel<T, OP><<<blocks, threads>>>(buf, iters, T(1));
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (e != cudaSuccess) return -1000;
    *rate = (double)blocks * threads * iters * CHAINS / (best * 1e-3);
    return 0;
}

}  // namespace

__global__ void div_kernel(int64_t n, const double *a, const double *b, double *q)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = k2::div_rn(a[i], b[i]);
}

__global__ void hypot_kernel(int64_t n, const double *a, const double *b, double *h)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = k2::hypot_cr(a[i], b[i]);
}

__global__ void hypotf_kernel(int64_t n, const float *a, const float *b, float *h)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = k2::hypot_cr(a[i], b[i]);
}

extern "C" int k2probe_hypotf(int64_t n, const float *a, const float *b, float *h, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!a || !b || !h) return -2;
    int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    hypotf_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, a, b, h);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1000;
}

extern "C" int k2probe_div(int64_t n, const double *a, const double *b, double *q, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!a || !b || !q) return -2;
    int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    div_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, a, b, q);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1000;
}

extern "C" int k2probe_hypot(int64_t n, const double *a, const double *b, double *h, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!a || !b || !h) return -2;
    int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    hypot_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, a, b, h);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1000;
}

__global__ void hypot_ncr_kernel(int64_t n, const double *a, const double *b, double *h)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = k2::hypot_ncr(a[i], b[i]);
}

__global__ void hypotf_ncr_kernel(int64_t n, const float *a, const float *b, float *h)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = k2::hypot_ncr(a[i], b[i]);
}

extern "C" int k2probe_hypot_ncr(int64_t n, const double *a, const double *b, double *h, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!a || !b || !h) return -2;
    int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    hypot_ncr_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, a, b, h);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1000;
}

extern "C" int k2probe_hypotf_ncr(int64_t n, const float *a, const float *b, float *h, void *stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!a || !b || !h) return -2;
    int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    hypotf_ncr_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, a, b, h);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1000;
}

extern "C" int k2probe_rate(int op, double *rate)
{
    switch (op) {
    case 0: return run<double, 0>(rate);
    case 1: return run<double, 1>(rate);
    case 2: return run<double, 2>(rate);
    case 3: return run<float, 0>(rate);
    case 4: return run<float, 1>(rate);
    case 5: return run<float, 2>(rate);
    default: return -1;
    }
}
