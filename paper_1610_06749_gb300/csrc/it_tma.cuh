// it_tma.cuh -- device helpers of the TMA-staged z-march kernels: mbarrier
// and TMA instructions (inline PTX), ring positions, the CTA's work
// segments and the paired-FP32 form of the cell update.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace itk {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// about 2^32 SM cycles (~2 s at 2 GHz) before a wait is declared lost
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 32)) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int xs, int y,
                                          int z) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(xs), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// a tensor map read from global memory: order its bytes (written before the
// launch) before the tensor-map proxy reads them
__device__ __forceinline__ void fence_tensormap_acquire(const void *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }


__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Position in the ring: slot index and the parity of its current phase.
struct RingPos {
    int slot;
    uint32_t phase;
    __device__ __forceinline__ void advance(int S) {
        if (++slot == S) { slot = 0; phase ^= 1u; }
    }
};

// The CTA's work: tile-planes (y-tile t, plane z) in the order t*nz + z,
// split into gridDim.x equal contiguous ranges.  A range is walked as
// segments (one tile column each); a segment computing planes [za, zb) loads
// planes za-1 .. zb.  The electrode ghost planes z = -1 and z = nz lie
// outside the tensor, and TMA fills them with zeros (n = 0 at the electrodes).
struct Segs {
    long long L, g1;
    int nz;
    int t, za, zb;
    __device__ __forceinline__ bool next() {
        if (L >= g1) return false;
        t = (int)(L / nz);
        za = (int)(L - (long long)t * nz);
        zb = (int)min((long long)nz, za + (g1 - L));
        L += zb - za;
        return true;
    }
    __device__ __forceinline__ int lo() const { return za - 1; }
    __device__ __forceinline__ int hi() const { return zb; }
};

// Plane n of a CTA's load sequence: its segments in order, each loading
// planes za-H .. zb+H-1 of its tile (H = 1 for one step per pass, 2 for two).
// Returns false past the end.
__device__ __forceinline__ bool plane_of(long long g0, long long g1, int nz, int n, int &t, int &z, int H = 1) {
    long long L = g0;
    while (L < g1) {
        const int tt = (int)(L / nz);
        const int za = (int)(L - (long long)tt * nz);
        const int zb = (int)min((long long)nz, za + (g1 - L));
        const int cnt = zb - za + 2 * H;
        if (n < cnt) {
            t = tt;
            z = za - H + n;
            return true;
        }
        n -= cnt;
        L += zb - za;
    }
    return false;
}

__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "r"(smem_u32(p)), "r"(v)
                 : "memory");
    return old;
}

// Four cells of upd7 (one float4 x-segment) with paired FP32 operations:
// each lane of a paired operation rounds exactly like the scalar operation
// (zm - n as fma(-1, n, zm), one rounding like the scalar subtraction), and
// the sequence is the one of upd7, so the results are bitwise those of the
// scalar kernels.
__device__ __forceinline__ float4 upd7x4(float4 n, float l, float r, float4 u, float4 d, float4 zm, float4 zp,
                                         float2 rxy, float2 rzw, float wd, float wzm, float wzp, float adt) {
    const float2 WD = make_float2(wd, wd), WZM = make_float2(wzm, wzm), WZP = make_float2(wzp, wzp);
    const float2 NA = make_float2(-adt, -adt), M4 = make_float2(-4.f, -4.f), M1 = make_float2(-1.f, -1.f);
    const float2 nxy = make_float2(n.x, n.y), nzw = make_float2(n.z, n.w);
    // x neighbours: cell x has (l, y), y has (x, z), z has (y, w), w has (z, r).
    // These pairs do not sit in aligned register pairs of the float4, so the
    // four sums are scalar (the same rounding as a paired add)
    const float2 xa = make_float2(__fadd_rn(l, n.y), __fadd_rn(n.x, n.z));
    const float2 xb = make_float2(__fadd_rn(n.y, n.w), __fadd_rn(n.z, r));
    const float2 sa = __fadd2_rn(xa, __fadd2_rn(make_float2(u.x, u.y), make_float2(d.x, d.y)));
    const float2 sb = __fadd2_rn(xb, __fadd2_rn(make_float2(u.z, u.w), make_float2(d.z, d.w)));
    float2 a = __fmul2_rn(WD, __ffma2_rn(M4, nxy, sa));
    float2 b = __fmul2_rn(WD, __ffma2_rn(M4, nzw, sb));
    a = __ffma2_rn(WZM, __ffma2_rn(M1, nxy, make_float2(zm.x, zm.y)), a);
    b = __ffma2_rn(WZM, __ffma2_rn(M1, nzw, make_float2(zm.z, zm.w)), b);
    a = __ffma2_rn(WZP, __ffma2_rn(M1, nxy, make_float2(zp.x, zp.y)), a);
    b = __ffma2_rn(WZP, __ffma2_rn(M1, nzw, make_float2(zp.z, zp.w)), b);
    a = __ffma2_rn(NA, rxy, a);
    b = __ffma2_rn(NA, rzw, b);
    a = __fadd2_rn(nxy, a);
    b = __fadd2_rn(nzw, b);
    return make_float4(a.x, a.y, b.x, b.y);
}

// The space-charge term of four cells (one float4), after upd7x4:
// v + sc n (n+ - n-), given d = n+ - n- as pairs (formed with a paired
// addition of -n-, which rounds like the scalar subtraction).  The same
// operation sequence as the scalar add_sc.  pxy/pzw receive n (n+ - n-), the
// tally of the term.
__device__ __forceinline__ float4 add_sc4(float4 v, float sc, float4 n, float2 dxy, float2 dzw, float2 &pxy,
                                          float2 &pzw) {
    const float2 SC = make_float2(sc, sc);
    pxy = __fmul2_rn(make_float2(n.x, n.y), dxy);
    pzw = __fmul2_rn(make_float2(n.z, n.w), dzw);
    const float2 a = __ffma2_rn(SC, pxy, make_float2(v.x, v.y));
    const float2 b = __ffma2_rn(SC, pzw, make_float2(v.z, v.w));
    return make_float4(a.x, a.y, b.x, b.y);
}

// n+ - n- of four cells as pairs
__device__ __forceinline__ void sc_diff4(float4 P, float4 M, float2 &dxy, float2 &dzw) {
    dxy = __fadd2_rn(make_float2(P.x, P.y), make_float2(-M.x, -M.y));
    dzw = __fadd2_rn(make_float2(P.z, P.w), make_float2(-M.z, -M.w));
}

}  // namespace itk
