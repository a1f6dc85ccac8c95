// Launch-shape helper shared by the kernels of libk2svd: persistent grids sized to the
// device (SM count x resident blocks per SM), so a grid-stride loop covers any batch.
#pragma once
#include <cuda_runtime.h>

#include "k2svd.h"

namespace k2 {

template <typename K>
static int grid_for(K kernel, int threads, size_t smem, int *blocks)
{
    int dev, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) return -1;
    if (per_sm < 1) per_sm = 1;
    *blocks = sms * per_sm;
    return 0;
}

// The entry points that copy a host-side table to the device (the n x n driver, its sigma
// gradient, the rectangular driver) refuse a stream that is being captured into a CUDA graph:
// a captured copy would read the host table when the graph is replayed, after the call has
// returned and the table is gone or reused.  Returns 0, K2SVD_ECAPTURE, or K2SVD_ECUDA when
// the stream cannot be queried.
static inline int capture_guard(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e == cudaErrorStreamCaptureImplicit) { cudaGetLastError(); return K2SVD_ECAPTURE; }
    if (e != cudaSuccess) return K2SVD_ECUDA;
    return cs == cudaStreamCaptureStatusNone ? 0 : K2SVD_ECAPTURE;
}

}  // namespace k2
