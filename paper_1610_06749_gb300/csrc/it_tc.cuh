// it_tc.cuh -- a bf16 GEMM on the 5th-generation tensor cores (tcgen05) for
// the surrogate network's matrix products.
//
//   D[m][n] = sum_k A[m][k] B[n][k]        (A, B bf16, K contiguous; D FP32)
//
// One CTA of 128 threads computes a 128 x 128 tile of D for one ensemble
// member (blockIdx.z):
//   * warp 0, one thread: TMA producer.  K is walked in chunks of 64
//     elements (128 bytes), each chunk of A (128 rows) and B (128 rows)
//     lands in one of four shared-memory stages with the 128-byte swizzle;
//   * warp 1, one thread: issues tcgen05.mma (M = 128, N = 128, K = 16,
//     kind::f16 with bf16 inputs and FP32 accumulation) from shared-memory
//     descriptors, accumulating in tensor memory, and hands each stage back
//     with tcgen05.commit once the MMAs reading it are done;
//   * warp 2 allocates (and at the end frees) 128 columns of tensor memory;
//   * all four warps then read the accumulator back with tcgen05.ld (warp w
//     owns TMEM lanes 32w .. 32w+31, i.e. rows 32w .. 32w+31 of the tile) and
//     run the epilogue functor on 32 x 32 blocks, each warp with a slice of
//     the (by then idle) stage memory to reorder its block for coalesced
//     stores.
// Every mbarrier wait is bounded (about 2^31 SM cycles); a wait that runs
// out raises the error flag, no further copy or MMA is issued, the copies
// already issued are waited for, and tensor memory is freed before return.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "it_tma.cuh"

namespace itk {
namespace tc {

constexpr int TM = 128, TN = 128, TK = 64, STAGES = 4;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
// dynamic shared memory: the stages (1024-byte aligned for the 128-byte
// swizzle) plus the alignment slack
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr long long WAIT_CYCLES = 1LL << 31;

// shared-memory matrix descriptor of a K-major tile with the 128-byte
// swizzle: start address / 16, leading-dimension offset 16 B (unused for
// this layout), stride between 8-row groups 1024 B, descriptor version 1,
// layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major,
// N = TN, M = TM
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tma_load3_cta(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// wait for phase `parity` of bar, at most WAIT_CYCLES; false if it ran out
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC), "r"(acc)
        : "memory");
}

// arrive on bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// D = A B^T for the tile (blockIdx.y, blockIdx.x) of member blockIdx.z; M,
// N: rows of D (TMA zero-fills the rows and the K tail outside the tensors;
// the epilogue masks rows >= M).  The whole warp calls
// epi(z, mw, lane, M, n0, v, scratch): lane holds D[mw + lane][n0 .. n0+31]
// in v, scratch is 32 x 33 floats of shared memory of this warp alone.
template <class Epi>
__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
               Epi epi, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *base = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.z, m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int nk = (K + TK - 1) / TK;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        failed = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    int issued = 0;   // chunks whose loads were issued (producer thread)
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            if (kc >= STAGES && !tc_wait(&empty[s], (uint32_t)((kc / STAGES - 1) & 1))) {
                failed = 1;
                break;
            }
            if (*(volatile int *)&failed) break;
            unsigned char *st = base + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load3_cta(st, &ta, &full[s], kc * TK, m0, z);
            tma_load3_cta(st + A_BYTES, &tb, &full[s], kc * TK, n0, z);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            if (!tc_wait(&full[s], (uint32_t)((kc / STAGES) & 1))) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(base + s * STAGE_BYTES), sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk)
                tc_mma(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), (kc | kk) != 0);
            tc_commit(&empty[s]);
        }
        // arrives once every MMA issued above has completed
        tc_commit(&done);
    }
    __syncwarp();
    // every thread: the accumulator is complete (or the run was abandoned)
    const bool ok = tc_wait(&done, 0u);
    tc_fence_after();
    if (!ok) failed = 1;
    __syncthreads();
    if (!failed) {
        // every copy has landed and every MMA has read its operands: the
        // stage memory is free for the epilogue's reordering
        float *scratch = reinterpret_cast<float *>(base) + warp * (32 * 33);
        const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < TN; c += 32) {
            float v[32];
            tc_ld32(row + (uint32_t)c, v);
            if (n0 + c < N) epi(z, m0 + warp * 32, lane, M, n0 + c, v, scratch);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0) {
        // no copy may be in flight when the CTA exits: the last load issued
        // into each stage has landed
        for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
            (void)tc_wait(&full[kc % STAGES], (uint32_t)((kc / STAGES) & 1));
        if (failed) atomicExch(err, 1);
    }
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

}  // namespace tc
}  // namespace itk
