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
//     halo row above and below, wrapped when the lateral faces are periodic.
//     Rows and planes outside the tensor (the absorbing faces' ghost rows, the
//     electrode ghost planes z = -1 and z = nz) are filled with zeros by TMA,
//     which is exactly the boundary condition n = 0;
//   * an S-deep ring of slots keeps S-2 planes in flight while one plane is
//     computed; the last warp to finish reading a slot refills it;
//   * each thread owns float4 x-segments and keeps their k-1 and k values in
//     registers; x and y neighbours and the k+1 plane come from shared memory;
//     the update runs on paired FP32 instructions (two cells per instruction);
//   * results are stored with coalesced 16-byte stores; per-thread FP32
//     partial sums (at most 32 planes) are reduced per warp in FP64 and per
//     CTA into the CTA's own tally slot (deterministic).
// Every mbarrier wait is bounded: a ring wait that runs out (after
// zc.wait_cycles SM cycles, 2^32 by default) raises the device error flag,
// and the CTA waits, with the full 2^32-cycle bound, for the copies it has
// issued and returns.  A test hook (zc.withhold) leaves the first ring load
// unissued, so that every warp's first wait runs out without any fault.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>

#include "it_device.cuh"
#include "it_internal.cuh"
#include "it_tma.cuh"

namespace itk {

struct ZmMaps {
    CUtensorMap main[2];   // n+, n- of the input set
    CUtensorMap halo[2];
};

constexpr int ZM_MAX_IPT = 4;                    // float4 items per thread
constexpr int ZM_MAX_SEG = 8;                    // segments of a CTA kept in shared memory

// Persistent step kernel: NW warps, all of them compute.
//   The planes a CTA needs stream through an S-deep ring of shared-memory
//   slots by TMA.  full[slot] completes when a plane's bytes have landed.
//   There is no producer warp: every warp, after its reads of a slot, adds
//   one to the slot's release counter, and the warp whose release completes
//   the count (the last reader) refills the slot with the plane S further
//   on.  So a slot is refilled the moment it is free, and all warps do the
//   same work.
//   Every warp marches up z, one plane per iteration, with no block-wide
//   barrier inside the march.  The FP64 tallies live in shared memory (each
//   warp's lane 0 adds to its own row), so the registers hold only the
//   marching planes and offsets.
template <bool PERIODIC, int IPT, int NW, bool SC>
__global__ void __launch_bounds__(NW * 32, (NW <= 8 ? 2 : 1))
step_zmarch_kernel(const __grid_constant__ ZmMaps maps, float *__restrict__ outp, float *__restrict__ outm,
                   int nx, int ny, int nz, const ZmConf zc, const Coef<float> cf, double *__restrict__ slots,
                   int *__restrict__ err) {
    constexpr int NT_ = NW * 32;
    extern __shared__ __align__(128) unsigned char zm_smem_raw[];
    // TMA destinations need 128-byte alignment: round the base up explicitly
    unsigned char *smem_base = zm_smem_raw + ((128u - (smem_u32(zm_smem_raw) & 127u)) & 127u);
    float *ring = reinterpret_cast<float *>(smem_base);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_base + (size_t)zc.S * zc.slot * sizeof(float));
    uint32_t *rel = reinterpret_cast<uint32_t *>(full + zc.S);   // release counters
    uint32_t *fills = rel + zc.S;                                  // loads issued per slot
    // per-warp FP64 tallies (tally q of warp w at w*WQ+q): 7 tallies, 9 with
    // space charge; a power-of-two row keeps the index a shift
    constexpr int WQ = SC ? 16 : 8, NQ = SC ? 9 : 7;
    __shared__ double wacc[NW * WQ];
    __shared__ volatile int abort_flag;
    __shared__ int seg_n0[ZM_MAX_SEG], seg_t[ZM_MAX_SEG], seg_za[ZM_MAX_SEG];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int ncol4 = nx >> 2;
    const int nitems = ncol4 * zc.TY;
    const int S = zc.S;
    const long long total = (long long)zc.ntile * nz;
    const long long g0 = total * blockIdx.x / gridDim.x;
    const long long g1 = total * (blockIdx.x + 1) / gridDim.x;

    // planes this CTA loads: every segment [za, zb) loads zb - za + 2.  The
    // first ZM_MAX_SEG segments are also kept in shared memory (first
    // sequence number, tile, za), so that a refill finds its plane without
    // the 64-bit divisions of the walk: a refill lies on the critical path,
    // since the warp that issues it is the last one done with the slot
    int nload = 0;
    int nseg = 0;
    {
        Segs sg{g0, g1, nz, 0, 0, 0};
        while (sg.next()) {
            if (tid == 0 && nseg < ZM_MAX_SEG) {
                seg_n0[nseg] = nload;
                seg_t[nseg] = sg.t;
                seg_za[nseg] = sg.za;
            }
            ++nseg;
            nload += sg.zb - sg.za + 2;
        }
    }
    const bool seg_cached = nseg <= ZM_MAX_SEG;

    // load plane n of the sequence into its slot (one thread)
    auto issue = [&](int n) {
        int t = 0, p = 0;
        if (n >= nload) return;
        if (seg_cached) {
            int i = 0;
            while (i + 1 < nseg && n >= seg_n0[i + 1]) ++i;
            t = seg_t[i];
            p = seg_za[i] - 1 + (n - seg_n0[i]);
        } else if (!plane_of(g0, g1, nz, n, t, p)) {
            return;
        }
        const int slot = n % S;
        const int y0 = t * zc.TY;
        // halo rows: wrapped when periodic; rows -1 and ny otherwise, which
        // lie outside the tensor and arrive as zeros (absorbing faces hold
        // n = 0); planes -1 and nz arrive as zeros the same way
        const int ytop = PERIODIC ? (y0 > 0 ? y0 - 1 : ny - 1) : y0 - 1;
        const int ybot = PERIODIC ? (y0 + zc.TY < ny ? y0 + zc.TY : 0) : y0 + zc.TY;
        const uint32_t tx = 2u * zc.nbx * (uint32_t)(zc.TY + 2) * zc.bx * 4u;
        float *base = ring + (size_t)slot * zc.slot;
        uint64_t *bar = &full[slot];
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, tx);
        for (int s = 0; s < 2; ++s) {
            if (zc.xs > 1) {
                // whole rows of a wide grid in one box (nbx == 1)
                float *blk = base + (size_t)s * zc.blk;
                tma_load4(blk + zc.reg_main, &maps.main[s], bar, 0, 0, y0, p);
                tma_load4(blk + zc.reg_top, &maps.halo[s], bar, 0, 0, ytop, p);
                tma_load4(blk + zc.reg_bot, &maps.halo[s], bar, 0, 0, ybot, p);
                continue;
            }
            for (int b = 0; b < zc.nbx; ++b) {
                float *blk = base + (size_t)(s * zc.nbx + b) * zc.blk;
                tma_load3(blk + zc.reg_main, &maps.main[s], bar, b * zc.bx, y0, p);
                tma_load3(blk + zc.reg_top, &maps.halo[s], bar, b * zc.bx, ytop, p);
                tma_load3(blk + zc.reg_bot, &maps.halo[s], bar, b * zc.bx, ybot, p);
            }
        }
        fills[slot] += 1;
    };

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            rel[q] = 0;
            fills[q] = 0;
        }
        for (int q = 0; q < NW * WQ; ++q) wacc[q] = 0.0;
        abort_flag = 0;
        fence_mbar_init();
        for (int n = zc.withhold ? 1 : 0; n < S && n < nload; ++n) issue(n);
    }
    __syncthreads();

    // warp-uniform: reduce one FP32 partial per lane in FP64 (fixed shuffle
    // order) and add it to the warp's tally q
    auto flush = [&](int q, float part) {
        double v = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wacc[warp * WQ + q] += v;
    };

    // per-item offsets inside a species block (species 1: + nbx*blk); x
    // neighbours are read from shared memory at wrapped offsets (periodic) or
    // replaced by zero at an absorbing row end
    int o_c[IPT], o_u[IPT], o_d[IPT], o_l[IPT], o_r[IPT], ty_[IPT], c4_[IPT];
    bool valid[IPT];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int q = tid + it * NT_;
        valid[it] = q < nitems;
        const int qe = valid[it] ? q : nitems - 1;
        const int ty = qe / ncol4, c4 = qe - (qe / ncol4) * ncol4;
        ty_[it] = ty;
        c4_[it] = c4;
        const int x0 = 4 * c4;
        const int xb = x0 / zc.bx, xi = x0 - xb * zc.bx;
        const int bofs = xb * zc.blk;
        o_c[it] = bofs + zc.reg_main + ty * zc.bx + xi;
        o_u[it] = bofs + (ty == 0 ? zc.reg_top : zc.reg_main + (ty - 1) * zc.bx) + xi;
        o_d[it] = bofs + (ty == zc.TY - 1 ? zc.reg_bot : zc.reg_main + (ty + 1) * zc.bx) + xi;
        const int xl = c4 == 0 ? nx - 1 : x0 - 1;
        const int xr = c4 == ncol4 - 1 ? 0 : x0 + 4;
        o_l[it] = (xl / zc.bx) * zc.blk + zc.reg_main + ty * zc.bx + (xl % zc.bx);
        o_r[it] = (xr / zc.bx) * zc.blk + zc.reg_main + ty * zc.bx + (xr % zc.bx);
    }
    const int sp_ofs = zc.nbx * zc.blk;
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
    RingPos pos{0, 0u};
    int nrel = 0;            // planes of the sequence this warp has released
    bool failed = false;

    // Wait (bounded by zc.wait_cycles) for the plane at ring position u.  A
    // lost wait marks the whole warp failed (shuffles stay convergent) and
    // raises the CTA's abort flag, after which no warp waits again.
    auto wait_full = [&](const RingPos &u) {
        if (failed) return;
        bool ok = mbar_try_wait(&full[u.slot], u.phase);
        if (__all_sync(0xffffffffu, ok)) return;
        const long long t0 = clock64();
        for (;;) {
            ok = ok || mbar_try_wait(&full[u.slot], u.phase);
            if (__all_sync(0xffffffffu, ok)) return;
            if (__any_sync(0xffffffffu, abort_flag || clock64() - t0 > zc.wait_cycles)) break;
        }
        failed = true;
        if (lane == 0) abort_flag = 1;
    };
    // After the warp's reads of the slot: count the release; the last of the
    // NW releases refills the slot.  A failed warp releases nothing, so no
    // slot is refilled while its previous load may still be in flight.
    auto release = [&](const RingPos &u) {
        __syncwarp();
        if (lane == 0 && !failed) {
            const uint32_t old = atom_add_acq_rel(&rel[u.slot], 1u);
            if (old % NW == NW - 1 && nrel + S < nload && !abort_flag) issue(nrel + S);
        }
        ++nrel;
    };

    Segs seg{g0, g1, nz, 0, 0, 0};
    while (seg.next()) {
        const int za = seg.za, zb = seg.zb;
        const int y0 = seg.t * zc.TY;
        float4 prev[IPT][2], cur[IPT][2];
        uint32_t off[IPT];       // element offset of the item in the current plane (cells < 2^32)
        bool edge_u[IPT], edge_d[IPT];   // rows at an absorbing y face (lateral tally)
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const int yg = y0 + ty_[it];
            off[it] = ((uint32_t)za * (uint32_t)ny + (uint32_t)yg) * (uint32_t)nx + 4u * (uint32_t)c4_[it];
            edge_u[it] = !PERIODIC && yg == 0;
            edge_d[it] = !PERIODIC && yg == ny - 1;
        }
        {
            wait_full(pos);
            const float *sl = ring + (size_t)pos.slot * zc.slot;
#pragma unroll
            for (int it = 0; it < IPT; ++it) {
                prev[it][0] = *reinterpret_cast<const float4 *>(sl + o_c[it]);
                prev[it][1] = *reinterpret_cast<const float4 *>(sl + sp_ofs + o_c[it]);
            }
            release(pos);
            pos.advance(S);
        }
        wait_full(pos);
        RingPos pc = pos;
        pos.advance(S);
        {
            const float *sl = ring + (size_t)pc.slot * zc.slot;
#pragma unroll
            for (int it = 0; it < IPT; ++it) {
                cur[it][0] = *reinterpret_cast<const float4 *>(sl + o_c[it]);
                cur[it][1] = *reinterpret_cast<const float4 *>(sl + sp_ofs + o_c[it]);
            }
        }
        float rsum = 0.f, lsum0 = 0.f, lsum1 = 0.f, ssum0 = 0.f, ssum1 = 0.f;
        int nacc = 0;
        // not unrolled: an unrolled march (which would save the register
        // rotation of prev/cur) measured slower
        for (int k = za; k < zb; ++k) {
            const bool electrode = k == 0 || k == nz - 1;
            wait_full(pos);
            const float *sk = ring + (size_t)pc.slot * zc.slot;
            const float *sn = ring + (size_t)pos.slot * zc.slot;
            float an[2] = {0.f, 0.f}, lat[2] = {0.f, 0.f};
#pragma unroll
            for (int it = 0; it < IPT; ++it) {
                const float4 P = cur[it][0], M = cur[it][1];
                const float2 rxy = __fmul2_rn(make_float2(P.x, P.y), make_float2(M.x, M.y));
                const float2 rzw = __fmul2_rn(make_float2(P.z, P.w), make_float2(M.z, M.w));
                float2 dxy, dzw;
                if (SC) sc_diff4(P, M, dxy, dzw);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float *bk = sk + s * sp_ofs;
                    const float4 n = cur[it][s];
                    const float4 u = *reinterpret_cast<const float4 *>(bk + o_u[it]);
                    const float4 d = *reinterpret_cast<const float4 *>(bk + o_d[it]);
                    const float4 zp = *reinterpret_cast<const float4 *>(sn + s * sp_ofs + o_c[it]);
                    float l = bk[o_l[it]];
                    float r = bk[o_r[it]];
                    if (!PERIODIC) {
                        if (c4_[it] == 0) l = 0.f;
                        if (c4_[it] == ncol4 - 1) r = 0.f;
                    }
                    float4 v = upd7x4(n, l, r, u, d, prev[it][s], zp, rxy, rzw,
                                      cf.wx[s], cf.wzm[s], cf.wzp[s], cf.adt);
                    if (SC) {
                        float2 pxy, pzw;
                        v = add_sc4(v, cf.sc[s], n, dxy, dzw, pxy, pzw);
                        if (valid[it]) (s ? ssum1 : ssum0) += (pxy.x + pxy.y) + (pzw.x + pzw.y);
                    }
                    if (valid[it]) {
                        *reinterpret_cast<float4 *>((s ? outm : outp) + off[it]) = v;
                        if (electrode) an[s] += (n.x + n.y) + (n.z + n.w);
                        if (!PERIODIC) {
                            if (c4_[it] == 0) lat[s] += n.x;
                            if (c4_[it] == ncol4 - 1) lat[s] += n.w;
                            if (edge_u[it]) lat[s] += (n.x + n.y) + (n.z + n.w);
                            if (edge_d[it]) lat[s] += (n.x + n.y) + (n.z + n.w);
                        }
                    }
                    prev[it][s] = n;
                    cur[it][s] = zp;
                }
                if (valid[it]) rsum += (rxy.x + rxy.y) + (rzw.x + rzw.y);
                off[it] += plane;
            }
            // FP32 partial sums over at most 32 planes, then FP64
            if (!PERIODIC) { lsum0 += lat[0]; lsum1 += lat[1]; }
            if (++nacc == 32) {
                flush(0, rsum);
                rsum = 0.f;
                if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); lsum0 = lsum1 = 0.f; }
                if (SC) { flush(7, ssum0); flush(8, ssum1); ssum0 = ssum1 = 0.f; }
                nacc = 0;
            }
            if (k == 0) { flush(1, an[0]); flush(2, an[1]); }
            if (k == nz - 1) { flush(3, an[0]); flush(4, an[1]); }
            release(pc);
            pc = pos;
            pos.advance(S);
        }
        flush(0, rsum);
        if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); }
        if (SC) { flush(7, ssum0); flush(8, ssum1); }
        release(pc);   // the plane zb above the segment
        if (failed) break;
    }
    if (failed && lane == 0) atomicExch(err, 1);
    __syncthreads();
    if (tid == 0) {
        // no load may be in flight when the CTA exits: wait (bounded) for the
        // last load issued into each slot (already complete unless a wait
        // was lost)
        for (int j = 0; j < S; ++j)
            if (fills[j] > 0) (void)mbar_wait_bounded(&full[j], (fills[j] - 1u) & 1u);
    }
    if (tid == 0 && !abort_flag) {
        double acc[NQ];
        for (int q = 0; q < NQ; ++q) {
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += wacc[w * WQ + q];
            acc[q] = t;
        }
        double *sl = slots + (size_t)blockIdx.x * NT;
        sl[0] += acc[0] * cf.rec_f;
        sl[1] += acc[1] * cf.anode_f[0];
        sl[2] += acc[2] * cf.anode_f[1];
        sl[3] += acc[3] * cf.cathode_f[0];
        sl[4] += acc[4] * cf.cathode_f[1];
        // lateral faces: x and y weights are equal for dx = dy (latx_f == laty_f)
        sl[5] += acc[5] * cf.latx_f[0];
        sl[6] += acc[6] * cf.latx_f[1];
        if (SC) {
            sl[7] += acc[NQ - 2] * cf.sc_f[0];
            sl[8] += acc[NQ - 1] * cf.sc_f[1];
        }
    }
}

}  // namespace itk

namespace itk {

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

int encode_map(CUtensorMap *m, void *base, int nx, int ny, int nz, int bx, int rows) {
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

// Wide rows (nx > 256, nx % 256 == 0): a 4-D view {256, nx / 256, ny, nz} of
// the same array (byte strides 1 KiB, one row, one plane), boxes of
// {256, nx / 256, rows, 1}, which land in shared memory as `rows` whole rows
// of nx floats: one copy per box where the 3-D view needs nx / 256.
int encode_map_rows(CUtensorMap *m, void *base, int nx, int ny, int nz, int rows) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return IT_ECUDA;
    }
    const int xs = nx / 256;
    cuuint64_t dims[4] = {256, (cuuint64_t)xs, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[3] = {256 * 4, (cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    cuuint32_t box[4] = {256, (cuuint32_t)xs, (cuuint32_t)rows, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (row view) failed (code " + std::to_string((int)r) + ")");
        return IT_ECUDA;
    }
    return IT_OK;
}

// bf16 operand of the tensor-core GEMM (it_tc.cuh): dims {K, rows, members}
// (K contiguous), byte strides of a row and of a member, boxes of 64 x 128
// with the 128-byte swizzle; rows and K beyond the dims arrive as zeros.
int encode_bf16_sw128(CUtensorMap *m, const void *base, long long K, long long rows, long long members,
                      long long row_bytes, long long member_bytes) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return IT_ECUDA;
    }
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)members};
    cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)member_bytes};
    cuuint32_t box[3] = {64, 128, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (bf16 operand) failed (code " + std::to_string((int)r) + ")");
        return IT_ECUDA;
    }
    return IT_OK;
}

static int align32f(int floats) { return (floats + 31) / 32 * 32; }   // 128-byte multiple of floats

// The dynamic shared-memory limit is a property of the kernel function,
// shared by every context: raise it to the device's opt-in maximum (never
// lower it to one context's need), so launches of other contexts with
// larger tiles stay valid.
template <bool P, int I, int W, bool S>
static cudaError_t zm_set_attr(size_t smem) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, step_zmarch_kernel<P, I, W, S>);
    if (e != cudaSuccess) return e;
    const int max_dyn = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the limit
    if ((int)smem > max_dyn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(step_zmarch_kernel<P, I, W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}

template <bool P, int I, int W, bool S>
static int zm_occupancy(size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_zmarch_kernel<P, I, W, S>, W * 32, smem) != cudaSuccess)
        return 0;
    return n;
}

static int ipt_of(const it_ctx *c, int TY, int nw) { return ((c->g.nx / 4) * TY + nw * 32 - 1) / (nw * 32); }

// Fill c->zm for a requested tile height / CTAs per SM / ring depth
// (0 = choose) and build the tensor maps.  One CTA per SM runs 16 warps,
// two CTAs per SM run 8 warps each.
int zmarch_setup(it_ctx *c, int want_ty, int want_cps, int want_s, int want_grid) {
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    if (c->prec != IT_FP32) { set_error("z-march kernel needs FP32 densities"); return IT_EINVAL; }
    if (nx % 4 != 0) { set_error("z-march kernel needs nx % 4 == 0"); return IT_EINVAL; }
    if (nx > 256 && nx % 256 != 0) { set_error("z-march kernel needs nx <= 256 or nx % 256 == 0"); return IT_EINVAL; }
    if ((unsigned long long)nx * ny * nz > 0xFFFFFFFFull) {
        set_error("z-march kernel indexes a species array with 32 bits: needs nx*ny*nz < 2^32");
        return IT_EINVAL;
    }
    const int cps = want_cps > 0 ? want_cps : 1;
    if (cps > 2) { set_error("z-march kernel runs 1 or 2 CTAs per SM"); return IT_EINVAL; }
    const int nw = cps == 1 ? 16 : 8;
    ZmConf z{};
    z.threads = nw * 32;
    // a ring block holds whole rows; rows wider than a TMA box dimension (256
    // floats) come through the 4-D view (nx / 256 pieces per row, one box)
    z.xs = nx > 256 ? nx / 256 : 1;
    z.bx = nx;
    z.nbx = 1;
    // rows per tile: the smallest divisor of ny that gives every thread two
    // float4 items (else the largest with at most ZM_MAX_IPT)
    int TY = want_ty;
    if (TY <= 0) {
        TY = 0;
        for (int t = 1; t <= ny; ++t) {
            if (ny % t) continue;
            if (ipt_of(c, t, nw) > ZM_MAX_IPT) break;
            TY = t;
            if ((nx / 4) * t >= 2 * z.threads) break;
        }
    }
    if (TY <= 0 || ny % TY != 0 || ipt_of(c, TY, nw) > ZM_MAX_IPT || TY > 255) {
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
    const size_t budget = (size_t)(220 * 1024) / cps;
    z.S = want_s > 0 ? want_s : 8;
    if (z.S < 3 || z.S > 16) { set_error("z-march ring depth must be 3..16"); return IT_EINVAL; }
    for (;;) {
        z.smem = (size_t)z.S * z.slot * sizeof(float) + 16 * z.S + 128;   // ring + barriers/counters + alignment slack
        if (z.smem <= budget || z.S == 3 || want_s > 0) break;
        --z.S;
    }
    if (z.smem > 227 * 1024) { set_error("z-march kernel: tile does not fit in shared memory"); return IT_EINVAL; }
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    const int ipt = ipt_of(c, TY, nw);
    cudaError_t e = cudaSuccess;
    int occ = 0;
    const bool sc = c->p.space_charge != 0;
#define ZM_CASE(P, I, W, S)                                        \
    if (per == P && ipt == I && nw == W && sc == S) {              \
        e = zm_set_attr<P, I, W, S>(z.smem);                       \
        occ = zm_occupancy<P, I, W, S>(z.smem);                    \
    }
#define ZM_CASES(S)                                                                          \
    ZM_CASE(true, 1, 16, S) ZM_CASE(true, 2, 16, S) ZM_CASE(true, 3, 16, S) ZM_CASE(true, 4, 16, S) \
    ZM_CASE(false, 1, 16, S) ZM_CASE(false, 2, 16, S) ZM_CASE(false, 3, 16, S) ZM_CASE(false, 4, 16, S) \
    ZM_CASE(true, 1, 8, S) ZM_CASE(true, 2, 8, S) ZM_CASE(true, 3, 8, S) ZM_CASE(true, 4, 8, S) \
    ZM_CASE(false, 1, 8, S) ZM_CASE(false, 2, 8, S) ZM_CASE(false, 3, 8, S) ZM_CASE(false, 4, 8, S)
    ZM_CASES(false) ZM_CASES(true)
#undef ZM_CASES
#undef ZM_CASE
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(z-march)");
    if (occ < cps) { set_error("z-march kernel: requested CTAs per SM do not fit"); return IT_EINVAL; }
    z.ctas_per_sm = cps;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // grid: CTAs, each taking one contiguous range of tile-planes.  0: one
    // per resident slot; -1: the largest multiple of the tile count that
    // fits the resident slots, so every tile column is cut at the same z and
    // vertically adjacent tiles are streamed in step (their halo rows are
    // then still in L2); > 0: as given.
    const long long tp = (long long)z.ntile * nz;
    long long grid = (long long)sms * cps;
    if (want_grid == -1 && grid >= z.ntile) grid = grid / z.ntile * z.ntile;
    else if (want_grid > 0) grid = want_grid;
    z.nzc = (int)std::min<long long>(grid, tp);
    for (int set = 0; set < 2; ++set)
        for (int s = 0; s < 2; ++s) {
            int rc = z.xs > 1 ? encode_map_rows(&c->tm_main[set][s], c->n[set][s], nx, ny, nz, TY)
                              : encode_map(&c->tm_main[set][s], c->n[set][s], nx, ny, nz, z.bx, TY);
            if (rc) return rc;
            rc = z.xs > 1 ? encode_map_rows(&c->tm_halo[set][s], c->n[set][s], nx, ny, nz, 1)
                          : encode_map(&c->tm_halo[set][s], c->n[set][s], nx, ny, nz, z.bx, 1);
            if (rc) return rc;
        }
    c->zm = z;
    c->zm_grid = z.nzc;
    return IT_OK;
}

int zmarch_configure(it_ctx *c) { return zmarch_setup(c, 0, 0, 0, 0); }

int launch_step_zmarch(it_ctx *c, cudaStream_t s) {
    const int cur = c->cur, nxt = cur ^ 1;
    ZmMaps maps;
    maps.main[0] = c->tm_main[cur][0];
    maps.main[1] = c->tm_main[cur][1];
    maps.halo[0] = c->tm_halo[cur][0];
    maps.halo[1] = c->tm_halo[cur][1];
    float *op = (float *)c->n[nxt][0], *om = (float *)c->n[nxt][1];
    ZmConf z = c->zm;
    z.wait_cycles = c->wait_cycles > 0 ? c->wait_cycles : (1LL << 32);
    z.withhold = c->withhold;
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    const int nw = z.threads / 32;
    const int ipt = ipt_of(c, z.TY, nw);
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    const bool sc = c->p.space_charge != 0;
#define ZM_LAUNCH(P, I, W, S)                                                                            \
    if (per == P && ipt == I && nw == W && sc == S)                                                      \
        step_zmarch_kernel<P, I, W, S><<<c->zm_grid, W * 32, z.smem, s>>>(maps, op, om, nx, ny, nz, z, c->cf, \
                                                                          c->d_slots, c->d_err);
#define ZM_LAUNCHES(S)                                                                                   \
    ZM_LAUNCH(true, 1, 16, S) ZM_LAUNCH(true, 2, 16, S) ZM_LAUNCH(true, 3, 16, S) ZM_LAUNCH(true, 4, 16, S) \
    ZM_LAUNCH(false, 1, 16, S) ZM_LAUNCH(false, 2, 16, S) ZM_LAUNCH(false, 3, 16, S) ZM_LAUNCH(false, 4, 16, S) \
    ZM_LAUNCH(true, 1, 8, S) ZM_LAUNCH(true, 2, 8, S) ZM_LAUNCH(true, 3, 8, S) ZM_LAUNCH(true, 4, 8, S) \
    ZM_LAUNCH(false, 1, 8, S) ZM_LAUNCH(false, 2, 8, S) ZM_LAUNCH(false, 3, 8, S) ZM_LAUNCH(false, 4, 8, S)
    ZM_LAUNCHES(false) ZM_LAUNCHES(true)
#undef ZM_LAUNCHES
#undef ZM_LAUNCH
    IT_CK(cudaGetLastError());
    c->cur = nxt;
    return IT_OK;
}

}  // namespace itk
