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

// One cell of the update as an increment in flux form:
//   n + [wd ((l + r) + (u + d) - 4 n) + wzm (zm - n) + wzp (zp - n) - adt rr]
// (wd = wx = wy: the cells are cubes).  Every transport term is a weight
// times a neighbour-minus-cell difference, so the transport part of the
// bracket sums to zero over the grid whatever the rounded weights: charge
// is moved, never made or lost, and each weight is simply its nearest FP32
// value.  The bracket's terms are small next to n, so their rounding errors
// are too; the one rounding of n + bracket is the only one at the scale of
// n.  The same operation sequence in every kernel, so all kernels round
// identically.
__device__ __forceinline__ float upd7(float n, float l, float r, float u, float d, float zm, float zp, float rr,
                                      float wd, float wzm, float wzp, float adt) {
    const float s4 = __fadd_rn(__fadd_rn(l, r), __fadd_rn(u, d));
    float v = __fmul_rn(wd, __fmaf_rn(-4.f, n, s4));
    v = __fmaf_rn(wzm, __fsub_rn(zm, n), v);
    v = __fmaf_rn(wzp, __fsub_rn(zp, n), v);
    v = __fmaf_rn(-adt, rr, v);
    return __fadd_rn(n, v);
}

__device__ __forceinline__ double upd7(double n, double l, double r, double u, double d, double zm, double zp,
                                       double rr, double wd, double wzm, double wzp, double adt) {
    const double s4 = __dadd_rn(__dadd_rn(l, r), __dadd_rn(u, d));
    double v = __dmul_rn(wd, __fma_rn(-4.0, n, s4));
    v = __fma_rn(wzm, __dsub_rn(zm, n), v);
    v = __fma_rn(wzp, __dsub_rn(zp, n), v);
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
