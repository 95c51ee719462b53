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

// One cell of the update in the increment form of Coef: n + [wc n + wx (l + r)
// + wy (u + d) + wzm zm + wzp zp - adt rr], the bracket's transport weights
// summing to zero (wc = w0 - 1).  The bracket's terms are a few percent of n,
// so their rounding errors are too, and the one rounding of n + bracket is
// the only one at the scale of n.  The same operation sequence in every
// kernel, so all kernels round identically.
__device__ __forceinline__ float upd7(float n, float l, float r, float u, float d, float zm, float zp, float rr,
                                      float wc, float wx, float wy, float wzm, float wzp, float adt) {
    float v = __fmul_rn(wc, n);
    v = __fmaf_rn(wx, __fadd_rn(l, r), v);
    v = __fmaf_rn(wy, __fadd_rn(u, d), v);
    v = __fmaf_rn(wzm, zm, v);
    v = __fmaf_rn(wzp, zp, v);
    v = __fmaf_rn(-adt, rr, v);
    return __fadd_rn(n, v);
}

__device__ __forceinline__ double upd7(double n, double l, double r, double u, double d, double zm, double zp,
                                       double rr, double wc, double wx, double wy, double wzm, double wzp,
                                       double adt) {
    double v = __dmul_rn(wc, n);
    v = __fma_rn(wx, __dadd_rn(l, r), v);
    v = __fma_rn(wy, __dadd_rn(u, d), v);
    v = __fma_rn(wzm, zm, v);
    v = __fma_rn(wzp, zp, v);
    v = __fma_rn(-adt, rr, v);
    return __dadd_rn(n, v);
}

// The space-charge term of one cell, after upd7: v + sc n (n+ - n-), in this
// operation order in every kernel (the paired form is add_sc4).
__device__ __forceinline__ float add_sc(float v, float sc, float n, float p, float m) {
    return __fmaf_rn(sc, __fmul_rn(n, __fsub_rn(p, m)), v);
}
__device__ __forceinline__ double add_sc(double v, double sc, double n, double p, double m) {
    return __fma_rn(sc, __dmul_rn(n, __dsub_rn(p, m)), v);
}

}  // namespace itk
