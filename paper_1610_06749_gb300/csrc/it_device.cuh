// it_device.cuh -- device helpers shared by the kernel files.
#pragma once

#include <cuda_runtime.h>

namespace itk {

// ---------------------------------------------------------------------------
// deterministic block reduction of N doubles (fixed shuffle and warp order)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double *smem /* [32][N] */) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) smem[warp * N + q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int q = 0; q < N; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += smem[w * N + q];
            v[q] = s;
        }
    }
}

}  // namespace itk
