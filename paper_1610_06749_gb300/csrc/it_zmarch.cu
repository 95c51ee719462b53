// it_zmarch.cu -- the bandwidth-bound step kernel for FP32 densities.
//
// One explicit step of the Appendix scheme for both species (Lax-Wendroff
// drift along z, 3-point diffusion on each axis, -alpha n+ n- from the old
// level; Eq. theEquation without space charge) with the electrode/lateral
// collection and recombination tallies fused in.
//
// Layout and data movement:
//   * a CTA owns TY full-width rows (y0 .. y0+TY-1) of one y-tile and marches
//     up a chunk of z planes [z0, z1);
//   * every plane it needs (z0-1 .. z1) arrives in a shared-memory slot by TMA
//     (cp.async.bulk.tensor, 3-D tiles of n+ and n-): TY main rows plus one
//     halo row above and below (wrapped when the lateral faces are periodic,
//     left at zero when they absorb); an S-deep ring of slots keeps S-2 planes
//     in flight while one plane is computed;
//   * each thread owns float4 x-segments and keeps their k-1 and k values in
//     registers; x neighbours come from warp shuffles, y neighbours and the
//     k+1 plane from shared memory;
//   * results are stored with coalesced 16-byte stores; per-thread FP32
//     partial sums per plane are accumulated in FP64 and reduced per CTA into
//     the CTA's own tally slot (deterministic).
// Every mbarrier wait is bounded: a wait that runs out raises the device
// error flag, waits (bounded) for the CTA's outstanding copies and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>

#include "it_device.cuh"
#include "it_internal.cuh"

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

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one cell of the flux-form update (same expression as the simple kernel)
__device__ __forceinline__ float upd(float n, float l, float r, float u, float d, float zm, float zp, float rr,
                                     float wx, float wy, float wzm, float wzp, float adt) {
    return n + wx * ((l - n) + (r - n)) + wy * ((u - n) + (d - n)) + wzm * (zm - n) + wzp * (zp - n) - adt * rr;
}

struct ZmMaps {
    CUtensorMap main[2];   // n+, n- of the input set
    CUtensorMap halo[2];
};

constexpr int ZM_THREADS = 256;
constexpr int ZM_MAX_IPT = 4;    // float4 items per thread

template <bool PERIODIC, int IPT>
__global__ void __launch_bounds__(ZM_THREADS)
step_zmarch_kernel(const __grid_constant__ ZmMaps maps, float *__restrict__ outp, float *__restrict__ outm,
                   int nx, int ny, int nz, const ZmConf zc, const Coef<float> cf, double *__restrict__ slots,
                   int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char zm_smem_raw[];
    // TMA destinations need 128-byte alignment: round the base up explicitly
    unsigned char *smem_base = zm_smem_raw + ((128u - (smem_u32(zm_smem_raw) & 127u)) & 127u);
    float *ring = reinterpret_cast<float *>(smem_base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_base + (size_t)zc.S * zc.slot * sizeof(float));
    __shared__ double red[32 * 7];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tile = blockIdx.x % zc.ntile;
    const int chunk = blockIdx.x / zc.ntile;
    const int y0 = tile * zc.TY;
    const int z0 = (int)(((long long)chunk * nz) / zc.nzc);
    const int z1 = (int)(((long long)(chunk + 1) * nz) / zc.nzc);
    const int zs = z0 > 0 ? z0 - 1 : 0;          // first plane loaded
    const int ze = z1 < nz ? z1 : nz - 1;         // last plane loaded
    const bool has_top = PERIODIC || y0 > 0;
    const bool has_bot = PERIODIC || y0 + zc.TY < ny;
    const int ytop = y0 > 0 ? y0 - 1 : ny - 1;
    const int ybot = y0 + zc.TY < ny ? y0 + zc.TY : 0;
    const uint32_t tx = 2u * zc.nbx * (uint32_t)(zc.TY + has_top + has_bot) * zc.bx * 4u;
    const int ncol4 = nx >> 2;
    const int nitems = ncol4 * zc.TY;

    if (tid == 0) {
        for (int q = 0; q < zc.S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    if (!(has_top && has_bot)) {
        // absorbing faces: halo rows outside the domain stay zero for the whole kernel
        for (int q = tid; q < zc.S * 2 * zc.nbx; q += ZM_THREADS) {
            float *blk = ring + (size_t)(q / (2 * zc.nbx)) * zc.slot + (size_t)(q % (2 * zc.nbx)) * zc.blk;
            for (int e = 0; e < zc.bx; ++e) {
                if (!has_top) blk[zc.reg_top + e] = 0.0f;
                if (!has_bot) blk[zc.reg_bot + e] = 0.0f;
            }
        }
    }
    fence_proxy_async();
    __syncthreads();

    // issue the TMA loads of plane p into its ring slot (thread 0 only)
    auto issue = [&](int p) {
        const int sl = (p - zs) % zc.S;
        float *base = ring + (size_t)sl * zc.slot;
        mbar_arrive_expect_tx(&bars[sl], tx);
        for (int s = 0; s < 2; ++s) {
            for (int b = 0; b < zc.nbx; ++b) {
                float *blk = base + (size_t)(s * zc.nbx + b) * zc.blk;
                tma_load3(blk + zc.reg_main, &maps.main[s], &bars[sl], b * zc.bx, y0, p);
                if (has_top) tma_load3(blk + zc.reg_top, &maps.halo[s], &bars[sl], b * zc.bx, ytop, p);
                if (has_bot) tma_load3(blk + zc.reg_bot, &maps.halo[s], &bars[sl], b * zc.bx, ybot, p);
            }
        }
    };
    auto slot_of = [&](int p) { return ring + (size_t)((p - zs) % zc.S) * zc.slot; };
    auto parity_of = [&](int p) { return (uint32_t)(((p - zs) / zc.S) & 1); };
    auto wait_plane = [&](int p) { return mbar_wait_bounded(&bars[(p - zs) % zc.S], parity_of(p)); };
    // pointer to row r (0 = top halo, 1..TY main, TY+1 bottom halo) of a block
    auto row_ptr = [&](const float *blk, int r) -> const float * {
        return blk + (r == 0 ? zc.reg_top : (r == zc.TY + 1 ? zc.reg_bot : zc.reg_main + (r - 1) * zc.bx));
    };

    int issued_hi = zs - 1;   // highest plane issued
    if (tid == 0) {
        for (int p = zs; p <= ze && p < zs + zc.S; ++p) issue(p);
    }
    issued_hi = min(ze, zs + zc.S - 1);

    // per-item coordinates
    int ity[IPT], ic4[IPT], ixb[IPT], ixi[IPT];
    bool ivalid[IPT];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int q = tid + it * ZM_THREADS;
        ivalid[it] = q < nitems;
        const int qe = ivalid[it] ? q : nitems - 1;
        ity[it] = qe / ncol4;
        ic4[it] = qe - ity[it] * ncol4;
        const int x0 = 4 * ic4[it];
        ixb[it] = x0 / zc.bx;
        ixi[it] = x0 - ixb[it] * zc.bx;
    }

    float4 prev[IPT][2], cur[IPT][2];
    bool failed = false;
    // centre values of plane p for every item
    auto load_centre = [&](int p, float4 (&dst)[IPT][2]) {
        const float *base = slot_of(p);
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float *blk = base + (size_t)(s * zc.nbx + ixb[it]) * zc.blk;
                dst[it][s] = *reinterpret_cast<const float4 *>(row_ptr(blk, ity[it] + 1) + ixi[it]);
            }
        }
    };

    // prologue: plane z0-1 (registers only) and plane z0
    if (z0 > 0) {
        failed |= !wait_plane(z0 - 1);
        load_centre(z0 - 1, prev);
    } else {
#pragma unroll
        for (int it = 0; it < IPT; ++it) prev[it][0] = prev[it][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    failed |= !wait_plane(z0);
    load_centre(z0, cur);
    if (__syncthreads_or(failed)) goto abort_path;
    if (z0 > 0 && issued_hi + 1 <= ze) {
        // the slot of plane z0-1 is free: refill it
        if (tid == 0) {
            fence_proxy_async();
            issue(issued_hi + 1);
        }
        ++issued_hi;
    }

    {
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = z0; k < z1; ++k) {
            const bool has_next = k + 1 <= nz - 1;
            if (has_next) failed |= !wait_plane(k + 1);
            {   // computed even after a lost wait (shuffles need the whole warp); stores are skipped
                const float *sk = slot_of(k);
                const float *sn = has_next ? slot_of(k + 1) : nullptr;
                float rsum = 0.f, an[2] = {0.f, 0.f}, ca[2] = {0.f, 0.f}, lx[2] = {0.f, 0.f}, ly[2] = {0.f, 0.f};
#pragma unroll
                for (int it = 0; it < IPT; ++it) {
                    const float4 P = cur[it][0], M = cur[it][1];
                    const float4 rr = make_float4(P.x * M.x, P.y * M.y, P.z * M.z, P.w * M.w);
                    const int ty = ity[it], c4 = ic4[it];
                    const int yg = y0 + ty;
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const float4 n = cur[it][s];
                        const float *blk = sk + (size_t)(s * zc.nbx + ixb[it]) * zc.blk;
                        const float4 u = *reinterpret_cast<const float4 *>(row_ptr(blk, ty) + ixi[it]);
                        const float4 d = *reinterpret_cast<const float4 *>(row_ptr(blk, ty + 2) + ixi[it]);
                        float4 zp = zero4;
                        if (has_next) {
                            const float *nb = sn + (size_t)(s * zc.nbx + ixb[it]) * zc.blk;
                            zp = *reinterpret_cast<const float4 *>(row_ptr(nb, ty + 1) + ixi[it]);
                        }
                        // x neighbours: shuffles within the row, shared memory at segment ends
                        float l = __shfl_up_sync(0xffffffffu, n.w, 1);
                        float r = __shfl_down_sync(0xffffffffu, n.x, 1);
                        if (c4 == 0) {
                            if (PERIODIC) {
                                const int xg = nx - 1;
                                const float *bb = sk + (size_t)(s * zc.nbx + xg / zc.bx) * zc.blk;
                                l = row_ptr(bb, ty + 1)[xg % zc.bx];
                            } else {
                                l = 0.f;
                            }
                        } else if (lane == 0) {
                            const int xg = 4 * c4 - 1;
                            const float *bb = sk + (size_t)(s * zc.nbx + xg / zc.bx) * zc.blk;
                            l = row_ptr(bb, ty + 1)[xg % zc.bx];
                        }
                        if (c4 == ncol4 - 1) {
                            if (PERIODIC) {
                                const float *bb = sk + (size_t)(s * zc.nbx) * zc.blk;
                                r = row_ptr(bb, ty + 1)[0];
                            } else {
                                r = 0.f;
                            }
                        } else if (lane == 31) {
                            const int xg = 4 * c4 + 4;
                            const float *bb = sk + (size_t)(s * zc.nbx + xg / zc.bx) * zc.blk;
                            r = row_ptr(bb, ty + 1)[xg % zc.bx];
                        }
                        const float4 zm = prev[it][s];
                        const float wx = cf.wx[s], wy = cf.wy[s], wzm = cf.wzm[s], wzp = cf.wzp[s], adt = cf.adt;
                        float4 v;
                        v.x = upd(n.x, l, n.y, u.x, d.x, zm.x, zp.x, rr.x, wx, wy, wzm, wzp, adt);
                        v.y = upd(n.y, n.x, n.z, u.y, d.y, zm.y, zp.y, rr.y, wx, wy, wzm, wzp, adt);
                        v.z = upd(n.z, n.y, n.w, u.z, d.z, zm.z, zp.z, rr.z, wx, wy, wzm, wzp, adt);
                        v.w = upd(n.w, n.z, r, u.w, d.w, zm.w, zp.w, rr.w, wx, wy, wzm, wzp, adt);
                        if (ivalid[it] && !failed) {
                            float *dst = (s ? outm : outp) + ((size_t)k * ny + yg) * nx + 4 * c4;
                            *reinterpret_cast<float4 *>(dst) = v;
                            const float nsum = (n.x + n.y) + (n.z + n.w);
                            if (k == 0) an[s] += nsum;
                            if (k == nz - 1) ca[s] += nsum;
                            if (!PERIODIC) {
                                if (c4 == 0) lx[s] += n.x;
                                if (c4 == ncol4 - 1) lx[s] += n.w;
                                if (yg == 0) ly[s] += nsum;
                                if (yg == ny - 1) ly[s] += nsum;
                            }
                        }
                        prev[it][s] = n;
                        cur[it][s] = zp;
                    }
                    if (ivalid[it]) rsum += (rr.x + rr.y) + (rr.z + rr.w);
                }
                acc[0] += (double)rsum;
                if (k == 0) { acc[1] += (double)an[0]; acc[2] += (double)an[1]; }
                if (k == nz - 1) { acc[3] += (double)ca[0]; acc[4] += (double)ca[1]; }
                if (!PERIODIC) {
                    acc[5] += (double)lx[0] * cf.latx_f[0] + (double)ly[0] * cf.laty_f[0];
                    acc[6] += (double)lx[1] * cf.latx_f[1] + (double)ly[1] * cf.laty_f[1];
                }
            }
            if (__syncthreads_or(failed)) goto abort_path;
            // slot of plane k is free: refill it with the next plane in order
            if (issued_hi + 1 <= ze) {
                if (tid == 0) {
                    fence_proxy_async();
                    issue(issued_hi + 1);
                }
                ++issued_hi;
            }
        }
        block_sum<7>(acc, red);
        if (tid == 0) {
            double *sl = slots + (size_t)blockIdx.x * NT;
            sl[0] += acc[0] * cf.rec_f;
            sl[1] += acc[1] * cf.anode_f[0];
            sl[2] += acc[2] * cf.anode_f[1];
            sl[3] += acc[3] * cf.cathode_f[0];
            sl[4] += acc[4] * cf.cathode_f[1];
            sl[5] += acc[5];
            sl[6] += acc[6];
        }
        return;
    }

abort_path:
    if (tid == 0) {
        atomicExch(err, 1);
        // wait (bounded) for every plane still in flight before the CTA exits
        for (int p = zs; p <= issued_hi; ++p) (void)mbar_wait_bounded(&bars[(p - zs) % zc.S], parity_of(p));
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// host side: launch shape and tensor maps
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static int encode_map(CUtensorMap *m, void *base, int nx, int ny, int nz, int bx, int rows) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return IT_ECUDA;
    }
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
        return IT_ECUDA;
    }
    return IT_OK;
}

static int align32f(int floats) { return (floats + 31) / 32 * 32; }   // 128-byte multiple of floats

template <bool P, int I>
static cudaError_t zm_set_attr(size_t smem) {
    return cudaFuncSetAttribute(step_zmarch_kernel<P, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <bool P, int I>
static int zm_occupancy(size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_zmarch_kernel<P, I>, ZM_THREADS, smem) != cudaSuccess)
        return 0;
    return n;
}

static int ipt_of(const it_ctx *c, int TY) { return ((c->g.nx / 4) * TY + ZM_THREADS - 1) / ZM_THREADS; }

// Fill c->zm for a requested TY / nzc / S (0 = choose) and build the maps.
int zmarch_setup(it_ctx *c, int want_ty, int want_nzc, int want_s) {
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    if (c->prec != IT_FP32) { set_error("z-march kernel needs FP32 densities"); return IT_EINVAL; }
    if (nx % 4 != 0) { set_error("z-march kernel needs nx % 4 == 0"); return IT_EINVAL; }
    if (nx > 256 && nx % 256 != 0) { set_error("z-march kernel needs nx <= 256 or nx % 256 == 0"); return IT_EINVAL; }
    ZmConf z{};
    z.threads = ZM_THREADS;
    z.bx = nx <= 256 ? nx : 256;
    z.nbx = nx / z.bx;
    // rows per tile: the smallest divisor of ny that gives every thread a
    // float4 item, with at most ZM_MAX_IPT items per thread
    int TY = want_ty;
    if (TY <= 0) {
        TY = 0;
        for (int t = 1; t <= ny; ++t) {
            if (ny % t) continue;
            if (ipt_of(c, t) > ZM_MAX_IPT) break;
            TY = t;
            if ((nx / 4) * t >= ZM_THREADS) break;
        }
    }
    if (TY <= 0 || ny % TY != 0 || ipt_of(c, TY) > ZM_MAX_IPT || TY > 255) {
        set_error("z-march kernel: no usable tile height for this grid");
        return IT_EINVAL;
    }
    z.TY = TY;
    z.ntile = ny / TY;
    z.reg_top = 0;
    z.reg_main = align32f(z.bx);
    z.reg_bot = z.reg_main + align32f(TY * z.bx);
    z.blk = z.reg_bot + align32f(z.bx);
    z.slot = 2 * z.nbx * z.blk;
    z.S = want_s > 0 ? want_s : 4;
    if (z.S < 3 || z.S > 8) { set_error("z-march ring depth must be 3..8"); return IT_EINVAL; }
    for (;;) {
        z.smem = (size_t)z.S * z.slot * sizeof(float) + 8 * 8 + 128;   // barriers + alignment slack
        if (z.smem <= 200 * 1024 || z.S == 3) break;
        --z.S;
    }
    if (z.smem > 227 * 1024) { set_error("z-march kernel: tile does not fit in shared memory"); return IT_EINVAL; }
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    const int ipt = ipt_of(c, TY);
    cudaError_t e = cudaSuccess;
    int occ = 0;
#define ZM_CASE(P, I) \
    if (per == P && ipt == I) { e = zm_set_attr<P, I>(z.smem); occ = zm_occupancy<P, I>(z.smem); }
    ZM_CASE(true, 1) ZM_CASE(true, 2) ZM_CASE(true, 3) ZM_CASE(true, 4)
    ZM_CASE(false, 1) ZM_CASE(false, 2) ZM_CASE(false, 3) ZM_CASE(false, 4)
#undef ZM_CASE
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(z-march)");
    if (occ < 1) { set_error("z-march kernel: zero occupancy"); return IT_EINVAL; }
    z.ctas_per_sm = occ;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nzc = want_nzc;
    if (nzc <= 0) {
        const int resident = sms * occ;
        nzc = std::max(1, resident / z.ntile);
        nzc = std::min(nzc, std::max(1, nz / 8));   // keep chunks at least ~8 planes deep
    }
    if (nzc > nz) nzc = nz;
    z.nzc = nzc;
    for (int set = 0; set < 2; ++set)
        for (int s = 0; s < 2; ++s) {
            int rc = encode_map(&c->tm_main[set][s], c->n[set][s], nx, ny, nz, z.bx, TY);
            if (rc) return rc;
            rc = encode_map(&c->tm_halo[set][s], c->n[set][s], nx, ny, nz, z.bx, 1);
            if (rc) return rc;
        }
    c->zm = z;
    c->zm_grid = z.ntile * z.nzc;
    return IT_OK;
}

int zmarch_configure(it_ctx *c) { return zmarch_setup(c, 0, 0, 0); }

int launch_step_zmarch(it_ctx *c, cudaStream_t s) {
    const int cur = c->cur, nxt = cur ^ 1;
    ZmMaps maps;
    maps.main[0] = c->tm_main[cur][0];
    maps.main[1] = c->tm_main[cur][1];
    maps.halo[0] = c->tm_halo[cur][0];
    maps.halo[1] = c->tm_halo[cur][1];
    float *op = (float *)c->n[nxt][0], *om = (float *)c->n[nxt][1];
    const ZmConf &z = c->zm;
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    const int ipt = ipt_of(c, z.TY);
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
#define ZM_LAUNCH(P, I)                                                                                 \
    if (per == P && ipt == I)                                                                           \
        step_zmarch_kernel<P, I><<<c->zm_grid, ZM_THREADS, z.smem, s>>>(maps, op, om, nx, ny, nz, z, c->cf, \
                                                                        c->d_slots, c->d_err);
    ZM_LAUNCH(true, 1) ZM_LAUNCH(true, 2) ZM_LAUNCH(true, 3) ZM_LAUNCH(true, 4)
    ZM_LAUNCH(false, 1) ZM_LAUNCH(false, 2) ZM_LAUNCH(false, 3) ZM_LAUNCH(false, 4)
#undef ZM_LAUNCH
    IT_CK(cudaGetLastError());
    c->cur = nxt;
    return IT_OK;
}

}  // namespace itk
