// Launch-shape helper shared by the kernels of libk2svd: persistent grids sized to the
// device (SM count x resident blocks per SM), so a grid-stride loop covers any batch.
#pragma once
#include <cuda_runtime.h>

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

}  // namespace k2
