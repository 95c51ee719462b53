// it_zmarch2.cu -- the step kernel with two time steps per pass (temporal
// blocking of depth 2) for FP32 densities.
//
// One launch advances the state by two explicit steps of the Appendix scheme
// (Eq. theEquation without space charge, the same weights and per-cell
// operation sequence as the one-step kernels, so the densities are bitwise
// those of two single steps), with the collection and recombination tallies
// of both steps fused in.  Each plane of the input is read from HBM once and
// each plane of the output written once, for two steps.
//
// A CTA owns TY full-width rows (y0 .. y0+TY-1) and marches up a chunk of z
// planes [za, zb):
//   * level t planes za-2 .. zb+1 stream through an S-deep ring by TMA, each
//     with two halo rows above and below (wrapped when periodic; rows outside
//     the tensor, and the planes -2, -1, nz, nz+1, arrive as zeros);
//   * at plane j the CTA computes the intermediate level t+1 on TY+2 rows
//     (its own rows and one halo row each side) into one of two shared-memory
//     planes, then, after a block barrier, level t+2 at plane j-1 from the
//     intermediate planes j-2, j-1, j (one block barrier per plane);
//   * the intermediate level is forced to zero where it is a ghost cell
//     (planes -1 and nz; rows -1 and ny when the lateral faces absorb);
//   * each thread owns one float4 x-segment of the tile and, for the halo
//     rows, threads 0 .. 2*nx/4-1 one more; the z history (level t at j-1, j
//     and the intermediate level at j-2, j-1) stays in registers;
//   * a ring slot is refilled by thread 0 after the block barrier that
//     follows its last reads.
// Tallies: first-step sums over the CTA's own rows at its own planes (the
// halo rows and planes are computed redundantly and not counted), second-step
// sums at the planes it writes; FP32 partials over at most 32 planes, FP64 per
// warp in shared memory, FP64 per CTA into its own slot.  Every mbarrier wait
// is bounded; a lost wait raises the device error flag.
#include <cudaTypedefs.h>

#include <algorithm>

#include "it_device.cuh"
#include "it_internal.cuh"
#include "it_tma.cuh"

namespace itk {

struct Zm2Maps {
    CUtensorMap main[2];   // n+, n- of the input set: TY rows
    CUtensorMap halo[2];   // two rows
};

template <bool PERIODIC, int NW, bool SC>
__global__ void __launch_bounds__(NW * 32, (NW <= 8 ? 2 : 1))
step_zmarch2_kernel(const __grid_constant__ Zm2Maps maps, float *__restrict__ outp, float *__restrict__ outm, int nx,
                    int ny, int nz, const Zm2Conf zc, const Coef<float> cf, double *__restrict__ slots,
                    int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char zm_smem_raw[];
    unsigned char *smem_base = zm_smem_raw + ((128u - (smem_u32(zm_smem_raw) & 127u)) & 127u);
    float *ring = reinterpret_cast<float *>(smem_base);
    float *mid = ring + (size_t)zc.S * zc.slot;   // two intermediate planes
    uint64_t *full = reinterpret_cast<uint64_t *>(mid + 2 * (size_t)zc.mslot);
    uint32_t *fills = reinterpret_cast<uint32_t *>(full + zc.S);   // loads issued per slot
    // per-warp FP64 tallies (tally q of warp w at w*WQ+q): 7 tallies, 9 with
    // space charge; a power-of-two row keeps the index a shift
    constexpr int WQ = SC ? 16 : 8, NQ = SC ? 9 : 7;
    __shared__ double wacc[NW * WQ];
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int ncol4 = nx >> 2;
    const int S = zc.S, TY = zc.TY, bx = zc.bx;
    const long long total = (long long)zc.ntile * nz;
    const long long g0 = total * blockIdx.x / gridDim.x;
    const long long g1 = total * (blockIdx.x + 1) / gridDim.x;

    // planes this CTA loads: every segment [za, zb) loads zb - za + 4
    int nload = 0;
    {
        Segs sg{g0, g1, nz, 0, 0, 0};
        while (sg.next()) nload += sg.zb - sg.za + 4;
    }

    // load plane n of the sequence into its slot (thread 0)
    auto issue = [&](int n) {
        int t = 0, p = 0;
        if (!plane_of(g0, g1, nz, n, t, p, 2)) return;
        const int slot = n % S;
        const int y0 = t * TY;
        const int ytop = PERIODIC ? (y0 >= 2 ? y0 - 2 : ny - 2) : y0 - 2;
        const int ybot = PERIODIC ? (y0 + TY < ny ? y0 + TY : 0) : y0 + TY;
        const uint32_t tx = 2u * zc.nbx * (uint32_t)(TY + 4) * bx * 4u;
        float *base = ring + (size_t)slot * zc.slot;
        uint64_t *bar = &full[slot];
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, tx);
        for (int s = 0; s < 2; ++s) {
            for (int b = 0; b < zc.nbx; ++b) {
                float *blk = base + (size_t)(s * zc.nbx + b) * zc.blk;
                tma_load3(blk + zc.reg_main, &maps.main[s], bar, b * bx, y0, p);
                tma_load3(blk + zc.reg_top, &maps.halo[s], bar, b * bx, ytop, p);
                tma_load3(blk + zc.reg_bot, &maps.halo[s], bar, b * bx, ybot, p);
            }
        }
        fills[slot] += 1;
    };

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            fills[q] = 0;
        }
        for (int q = 0; q < NW * WQ; ++q) wacc[q] = 0.0;
        abort_flag = 0;
        fence_mbar_init();
        for (int n = 0; n < S && n < nload; ++n) issue(n);
    }
    __syncthreads();

    auto flush = [&](int q, float part) {
        double v = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wacc[warp * WQ + q] += v;
    };
    // offset of ring row r (y = y0 - 2 + r) in a block
    auto rrow = [&](int r) {
        return r < 2 ? zc.reg_top + r * bx : (r < TY + 2 ? zc.reg_main + (r - 2) * bx : zc.reg_bot + (r - TY - 2) * bx);
    };

    // own item: output row o (y = y0 + o), float4 column c4
    const int o = tid / ncol4, c4 = tid - (tid / ncol4) * ncol4;
    const int x0 = 4 * c4;
    const int xl = c4 == 0 ? nx - 1 : x0 - 1, xr = c4 == ncol4 - 1 ? 0 : x0 + 4;
    const int r_o = rrow(o + 2);
    const int t_c = (x0 / bx) * zc.blk + r_o + x0 % bx;                 // level t, ring
    const int t_u = (x0 / bx) * zc.blk + rrow(o + 1) + x0 % bx;
    const int t_d = (x0 / bx) * zc.blk + rrow(o + 3) + x0 % bx;
    const int t_l = (xl / bx) * zc.blk + r_o + xl % bx;
    const int t_r = (xr / bx) * zc.blk + r_o + xr % bx;
    const int m_c = (x0 / bx) * zc.mblk + (o + 1) * bx + x0 % bx;      // intermediate plane, row o+1
    const int m_l = (xl / bx) * zc.mblk + (o + 1) * bx + xl % bx;
    const int m_r = (xr / bx) * zc.mblk + (o + 1) * bx + xr % bx;
    const bool zero_l = !PERIODIC && c4 == 0, zero_r = !PERIODIC && c4 == ncol4 - 1;
    // halo item (threads below 2*ncol4): intermediate row 0 (y0 - 1) or TY+1 (y0 + TY)
    const bool has_h = tid < 2 * ncol4;
    const int hq = has_h ? tid : 0;
    const bool h_top = hq < ncol4;
    const int hc4 = h_top ? hq : hq - ncol4;
    const int hx0 = 4 * hc4;
    const int hxl = hc4 == 0 ? nx - 1 : hx0 - 1, hxr = hc4 == ncol4 - 1 ? 0 : hx0 + 4;
    const int hr = h_top ? 1 : TY + 2;                                     // ring row of the halo item
    const int h_c = (hx0 / bx) * zc.blk + rrow(hr) + hx0 % bx;
    const int h_u = (hx0 / bx) * zc.blk + rrow(hr - 1) + hx0 % bx;
    const int h_d = (hx0 / bx) * zc.blk + rrow(hr + 1) + hx0 % bx;
    const int h_l = (hxl / bx) * zc.blk + rrow(hr) + hxl % bx;
    const int h_r = (hxr / bx) * zc.blk + rrow(hr) + hxr % bx;
    const int h_m = (hx0 / bx) * zc.mblk + (h_top ? 0 : TY + 1) * bx + hx0 % bx;
    const bool hzero_l = !PERIODIC && hc4 == 0, hzero_r = !PERIODIC && hc4 == ncol4 - 1;

    const int rsp = zc.nbx * zc.blk;    // species offset in a ring slot
    const int msp = zc.nbx * zc.mblk;   // species offset in an intermediate plane
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    bool failed = false;
    RingPos pos{0, 0u};       // ring position of the next plane to wait for
    int released = 0;         // thread 0: planes of the sequence handed back so far
    int seq0 = 0;             // sequence index of the current segment's first plane

    // bounded wait for the plane at ring position u (every thread)
    auto wait_full = [&](const RingPos &u) {
        if (failed) return;
        bool ok = mbar_try_wait(&full[u.slot], u.phase);
        if (__all_sync(0xffffffffu, ok)) return;
        const long long t0 = clock64();
        for (;;) {
            ok = ok || mbar_try_wait(&full[u.slot], u.phase);
            if (__all_sync(0xffffffffu, ok)) return;
            if (__any_sync(0xffffffffu, abort_flag || clock64() - t0 > (1LL << 32))) break;
        }
        failed = true;
        if (lane == 0) abort_flag = 1;
    };
    // thread 0, after a block barrier: refill every slot whose plane (sequence
    // index < upto) every thread has finished reading.  A slot whose load has
    // not completed (only after a lost wait) is not refilled.
    auto release_upto = [&](int upto) {
        while (released < upto) {
            const int slot = released % S;
            const uint32_t ph = (uint32_t)(released / S) & 1u;
            if (abort_flag || !mbar_test_wait(&full[slot], ph)) {
                abort_flag = 1;
                released = upto;
                break;
            }
            if (released + S < nload) issue(released + S);
            ++released;
        }
    };

    Segs seg{g0, g1, nz, 0, 0, 0};
    while (seg.next()) {
        const int za = seg.za, zb = seg.zb;
        const int y0 = seg.t * TY;
        const int yo = y0 + o;
        const bool edge_y = !PERIODIC && (yo == 0 || yo == ny - 1);
        const bool h_in = PERIODIC || (h_top ? y0 >= 1 : y0 + TY < ny);   // the halo row is inside the domain
        uint32_t off = ((uint32_t)za * (uint32_t)ny + (uint32_t)yo) * (uint32_t)nx + (uint32_t)x0;   // plane za
        float4 Tp[2], Tc[2], Hp[2], Hc[2], Mm2[2], Mm1[2];
        // level t at planes za-2 and za-1
        RingPos pj;
        wait_full(pos);
        {
            const float *sl = ring + (size_t)pos.slot * zc.slot;
            Tp[0] = *reinterpret_cast<const float4 *>(sl + t_c);
            Tp[1] = *reinterpret_cast<const float4 *>(sl + rsp + t_c);
            Hp[0] = *reinterpret_cast<const float4 *>(sl + h_c);
            Hp[1] = *reinterpret_cast<const float4 *>(sl + rsp + h_c);
        }
        pos.advance(S);
        wait_full(pos);
        {
            const float *sl = ring + (size_t)pos.slot * zc.slot;
            Tc[0] = *reinterpret_cast<const float4 *>(sl + t_c);
            Tc[1] = *reinterpret_cast<const float4 *>(sl + rsp + t_c);
            Hc[0] = *reinterpret_cast<const float4 *>(sl + h_c);
            Hc[1] = *reinterpret_cast<const float4 *>(sl + rsp + h_c);
        }
        pj = pos;
        pos.advance(S);
        Mm2[0] = Mm2[1] = Mm1[0] = Mm1[1] = zero4;
        float rsum = 0.f, lsum0 = 0.f, lsum1 = 0.f, ssum0 = 0.f, ssum1 = 0.f;
        int nacc = 0;
        for (int j = za - 1; j <= zb; ++j) {
            wait_full(pos);   // level t at plane j+1
            const float *sj = ring + (size_t)pj.slot * zc.slot;
            const float *sn = ring + (size_t)pos.slot * zc.slot;
            const bool jin = j >= 0 && j < nz;
            const bool own = j >= za && j < zb;
            // electrode sums of the first step (plane j) and the second (plane j-1)
            float an1[2] = {0.f, 0.f}, an2[2] = {0.f, 0.f}, lat[2] = {0.f, 0.f};
            // ---- first step: intermediate level at plane j ----
            float4 Mj[2], Hm[2];
            {
                const float2 rxy = __fmul2_rn(make_float2(Tc[0].x, Tc[0].y), make_float2(Tc[1].x, Tc[1].y));
                const float2 rzw = __fmul2_rn(make_float2(Tc[0].z, Tc[0].w), make_float2(Tc[1].z, Tc[1].w));
                float2 dxy, dzw;
                if (SC) sc_diff4(Tc[0], Tc[1], dxy, dzw);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float *bk = sj + s * rsp;
                    const float4 u = *reinterpret_cast<const float4 *>(bk + t_u);
                    const float4 d = *reinterpret_cast<const float4 *>(bk + t_d);
                    const float4 zp = *reinterpret_cast<const float4 *>(sn + s * rsp + t_c);
                    float l = bk[t_l], r = bk[t_r];
                    if (zero_l) l = 0.f;
                    if (zero_r) r = 0.f;
                    float4 v = upd7x4(Tc[s], l, r, u, d, Tp[s], zp, rxy, rzw, cf.wx[s], cf.wzm[s], cf.wzp[s], cf.adt);
                    if (SC) {
                        float2 pxy, pzw;
                        v = add_sc4(v, cf.sc[s], Tc[s], dxy, dzw, pxy, pzw);
                        if (own) (s ? ssum1 : ssum0) += (pxy.x + pxy.y) + (pzw.x + pzw.y);
                    }
                    Mj[s] = jin ? v : zero4;
                    if (own) {
                        const float4 n = Tc[s];
                        if (j == 0 || j == nz - 1) an1[s] += (n.x + n.y) + (n.z + n.w);
                        if (!PERIODIC) {
                            if (c4 == 0) lat[s] += n.x;
                            if (c4 == ncol4 - 1) lat[s] += n.w;
                            if (edge_y) lat[s] += (n.x + n.y) + (n.z + n.w);
                        }
                    }
                    Tp[s] = Tc[s];
                    Tc[s] = zp;
                }
                if (own) rsum += (rxy.x + rxy.y) + (rzw.x + rzw.y);
            }
            if (has_h) {
                const float2 rxy = __fmul2_rn(make_float2(Hc[0].x, Hc[0].y), make_float2(Hc[1].x, Hc[1].y));
                const float2 rzw = __fmul2_rn(make_float2(Hc[0].z, Hc[0].w), make_float2(Hc[1].z, Hc[1].w));
                float2 dxy, dzw;
                if (SC) sc_diff4(Hc[0], Hc[1], dxy, dzw);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float *bk = sj + s * rsp;
                    const float4 u = *reinterpret_cast<const float4 *>(bk + h_u);
                    const float4 d = *reinterpret_cast<const float4 *>(bk + h_d);
                    const float4 zp = *reinterpret_cast<const float4 *>(sn + s * rsp + h_c);
                    float l = bk[h_l], r = bk[h_r];
                    if (hzero_l) l = 0.f;
                    if (hzero_r) r = 0.f;
                    float4 v = upd7x4(Hc[s], l, r, u, d, Hp[s], zp, rxy, rzw, cf.wx[s], cf.wzm[s], cf.wzp[s], cf.adt);
                    if (SC) {
                        float2 pxy, pzw;
                        v = add_sc4(v, cf.sc[s], Hc[s], dxy, dzw, pxy, pzw);   // halo: not tallied
                    }
                    Hm[s] = (jin && h_in) ? v : zero4;
                    Hp[s] = Hc[s];
                    Hc[s] = zp;
                }
            }
            // One barrier per plane: every thread has finished the previous
            // second step (which read the intermediate plane that plane j now
            // overwrites) and its reads of level t plane j; the writes of
            // plane j below are read after the next plane's barrier.
            __syncthreads();
            if (tid == 0) release_upto(seq0 + (j - za + 2) + 1);
            {
                float *mb = mid + (size_t)(j & 1) * zc.mslot;
                *reinterpret_cast<float4 *>(mb + m_c) = Mj[0];
                *reinterpret_cast<float4 *>(mb + msp + m_c) = Mj[1];
                if (has_h) {
                    *reinterpret_cast<float4 *>(mb + h_m) = Hm[0];
                    *reinterpret_cast<float4 *>(mb + msp + h_m) = Hm[1];
                }
            }
            // ---- second step: level t+2 at plane j-1 ----
            if (j - 1 >= za) {
                const float *mb = mid + (size_t)((j - 1) & 1) * zc.mslot;
                const float2 rxy = __fmul2_rn(make_float2(Mm1[0].x, Mm1[0].y), make_float2(Mm1[1].x, Mm1[1].y));
                const float2 rzw = __fmul2_rn(make_float2(Mm1[0].z, Mm1[0].w), make_float2(Mm1[1].z, Mm1[1].w));
                float2 dxy, dzw;
                if (SC) sc_diff4(Mm1[0], Mm1[1], dxy, dzw);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float *bk = mb + s * msp;
                    const float4 u = *reinterpret_cast<const float4 *>(bk + m_c - bx);
                    const float4 d = *reinterpret_cast<const float4 *>(bk + m_c + bx);
                    float l = bk[m_l], r = bk[m_r];
                    if (zero_l) l = 0.f;
                    if (zero_r) r = 0.f;
                    float4 v = upd7x4(Mm1[s], l, r, u, d, Mm2[s], Mj[s], rxy, rzw,
                                      cf.wx[s], cf.wzm[s], cf.wzp[s], cf.adt);
                    if (SC) {
                        float2 pxy, pzw;
                        v = add_sc4(v, cf.sc[s], Mm1[s], dxy, dzw, pxy, pzw);
                        (s ? ssum1 : ssum0) += (pxy.x + pxy.y) + (pzw.x + pzw.y);
                    }
                    *reinterpret_cast<float4 *>((s ? outm : outp) + off) = v;
                    const float4 n = Mm1[s];
                    if (j - 1 == 0 || j - 1 == nz - 1) an2[s] += (n.x + n.y) + (n.z + n.w);
                    if (!PERIODIC) {
                        if (c4 == 0) lat[s] += n.x;
                        if (c4 == ncol4 - 1) lat[s] += n.w;
                        if (edge_y) lat[s] += (n.x + n.y) + (n.z + n.w);
                    }
                }
                rsum += (rxy.x + rxy.y) + (rzw.x + rzw.y);
                off += plane;
            }
            Mm2[0] = Mm1[0]; Mm2[1] = Mm1[1];
            Mm1[0] = Mj[0]; Mm1[1] = Mj[1];
            // tallies: FP32 partials over at most 32 planes, then FP64
            if (!PERIODIC) { lsum0 += lat[0]; lsum1 += lat[1]; }
            if (++nacc == 32) {
                flush(0, rsum);
                rsum = 0.f;
                if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); lsum0 = lsum1 = 0.f; }
                if (SC) { flush(7, ssum0); flush(8, ssum1); ssum0 = ssum1 = 0.f; }
                nacc = 0;
            }
            // anode: plane 0, cathode: plane nz-1, of either step
            if (own && j == 0) { flush(1, an1[0]); flush(2, an1[1]); }
            if (own && j == nz - 1) { flush(3, an1[0]); flush(4, an1[1]); }
            if (j - 1 >= za && j - 1 == 0) { flush(1, an2[0]); flush(2, an2[1]); }
            if (j - 1 >= za && j - 1 == nz - 1) { flush(3, an2[0]); flush(4, an2[1]); }
            pj = pos;
            pos.advance(S);
        }
        flush(0, rsum);
        if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); }
        if (SC) { flush(7, ssum0); flush(8, ssum1); }
        seq0 += zb - za + 4;
        // hand back plane zb+1 too: the next segment waits for its first three
        // planes before its first barrier, and with S = 3 one of them goes
        // into this slot
        __syncthreads();
        if (tid == 0) release_upto(seq0);
    }
    if (failed && lane == 0) atomicExch(err, 1);
    __syncthreads();
    if (tid == 0) {
        // no load may be in flight when the CTA exits: wait (bounded) for the
        // last load issued into each slot
        for (int q = 0; q < S; ++q)
            if (fills[q] > 0) (void)mbar_wait_bounded(&full[q], (fills[q] - 1u) & 1u);
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
        sl[5] += acc[5] * cf.latx_f[0];
        sl[6] += acc[6] * cf.latx_f[1];
        if (SC) {
            sl[7] += acc[NQ - 2] * cf.sc_f[0];
            sl[8] += acc[NQ - 1] * cf.sc_f[1];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int align32f2(int floats) { return (floats + 31) / 32 * 32; }

template <bool P, int W, bool S>
static cudaError_t zm2_set_attr(size_t smem, int *occ) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, step_zmarch2_kernel<P, W, S>);
    if (e != cudaSuccess) return e;
    const int max_dyn = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the limit
    if ((int)smem > max_dyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(step_zmarch2_kernel<P, W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step_zmarch2_kernel<P, W, S>, W * 32, smem);
}

// Fill c->zm2 for a tile height / CTAs per SM / ring depth / grid rule (0 =
// choose).  One CTA per SM runs 16 warps, two run 8 warps each; every thread
// owns one float4 of the tile, so TY = threads / (nx / 4).
int zmarch2_setup(it_ctx *c, int want_ty, int want_cps, int want_s, int want_grid) {
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    if (c->prec != IT_FP32) { set_error("z-march kernels need FP32 densities"); return IT_EINVAL; }
    if (nx % 4 != 0) { set_error("z-march kernels need nx % 4 == 0"); return IT_EINVAL; }
    if (nx > 256 && nx % 256 != 0) { set_error("z-march kernels need nx <= 256 or nx % 256 == 0"); return IT_EINVAL; }
    if ((unsigned long long)nx * ny * nz > 0xFFFFFFFFull) {
        set_error("z-march kernels index a species array with 32 bits: needs nx*ny*nz < 2^32");
        return IT_EINVAL;
    }
    const int ncol4 = nx / 4;
    // default: two CTAs of 8 warps per SM where that tile fits the grid, else one of 16
    int cps = want_cps;
    if (cps <= 0) cps = (256 % ncol4 == 0 && 2 * ncol4 <= 256 && ny % (256 / ncol4) == 0) ? 2 : 1;
    if (cps > 2) { set_error("the two-step z-march kernel runs 1 or 2 CTAs per SM"); return IT_EINVAL; }
    const int nw = cps == 1 ? 16 : 8;
    const int threads = nw * 32;
    if (threads % ncol4 != 0 || 2 * ncol4 > threads) {
        set_error("two-step z-march kernel: one float4 per thread needs (nx/4) to divide the CTA's threads");
        return IT_EINVAL;
    }
    const int TY = threads / ncol4;
    if (want_ty > 0 && want_ty != TY) {
        set_error("two-step z-march kernel: the tile height is threads / (nx/4) = " + std::to_string(TY));
        return IT_EINVAL;
    }
    if (ny % TY != 0 || ny < 4 || TY + 4 > 256) {
        set_error("two-step z-march kernel: ny must be a multiple of the tile height " + std::to_string(TY));
        return IT_EINVAL;
    }
    Zm2Conf z{};
    z.threads = threads;
    z.TY = TY;
    z.ntile = ny / TY;
    z.bx = nx <= 256 ? nx : 256;
    z.nbx = nx / z.bx;
    z.reg_top = 0;
    z.reg_main = align32f2(2 * z.bx);
    z.reg_bot = z.reg_main + align32f2(TY * z.bx);
    z.blk = z.reg_bot + align32f2(2 * z.bx);
    z.slot = 2 * z.nbx * z.blk;
    z.mblk = align32f2((TY + 2) * z.bx);
    z.mslot = 2 * z.nbx * z.mblk;
    const size_t budget = (size_t)(220 * 1024) / cps;
    z.S = want_s > 0 ? want_s : 6;
    if (z.S < 3 || z.S > 16) { set_error("z-march ring depth must be 3..16"); return IT_EINVAL; }
    for (;;) {
        z.smem = ((size_t)z.S * z.slot + 2 * (size_t)z.mslot) * sizeof(float) + 16 * z.S + 128;
        if (z.smem <= budget || z.S == 3 || want_s > 0) break;
        --z.S;
    }
    if (z.smem > 227 * 1024) { set_error("two-step z-march kernel: tile does not fit in shared memory"); return IT_EINVAL; }
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    cudaError_t e = cudaSuccess;
    int occ = 0;
    const bool sc = c->p.space_charge != 0;
    if (per && nw == 16) e = sc ? zm2_set_attr<true, 16, true>(z.smem, &occ) : zm2_set_attr<true, 16, false>(z.smem, &occ);
    if (per && nw == 8) e = sc ? zm2_set_attr<true, 8, true>(z.smem, &occ) : zm2_set_attr<true, 8, false>(z.smem, &occ);
    if (!per && nw == 16) e = sc ? zm2_set_attr<false, 16, true>(z.smem, &occ) : zm2_set_attr<false, 16, false>(z.smem, &occ);
    if (!per && nw == 8) e = sc ? zm2_set_attr<false, 8, true>(z.smem, &occ) : zm2_set_attr<false, 8, false>(z.smem, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(two-step z-march)");
    if (occ < cps) { set_error("two-step z-march kernel: requested CTAs per SM do not fit"); return IT_EINVAL; }
    z.ctas_per_sm = cps;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // grid rules as for the one-step kernel: 0 = one CTA per resident slot,
    // -1 = the largest multiple of the tile count that fits, > 0 = as given
    const long long tp = (long long)z.ntile * nz;
    long long grid = (long long)sms * cps;
    if (want_grid == -1 && grid >= z.ntile) grid = grid / z.ntile * z.ntile;
    else if (want_grid > 0) grid = want_grid;
    z.grid = (int)std::min<long long>(grid, tp);
    for (int set = 0; set < 2; ++set)
        for (int s = 0; s < 2; ++s) {
            int rc = encode_map(&c->tm_main2[set][s], c->n[set][s], nx, ny, nz, z.bx, TY);
            if (rc) return rc;
            rc = encode_map(&c->tm_halo2[set][s], c->n[set][s], nx, ny, nz, z.bx, 2);
            if (rc) return rc;
        }
    c->zm2 = z;
    return IT_OK;
}

// two explicit steps in one launch
int launch_step_zmarch2(it_ctx *c, cudaStream_t s) {
    const int cur = c->cur, nxt = cur ^ 1;
    Zm2Maps maps;
    maps.main[0] = c->tm_main2[cur][0];
    maps.main[1] = c->tm_main2[cur][1];
    maps.halo[0] = c->tm_halo2[cur][0];
    maps.halo[1] = c->tm_halo2[cur][1];
    float *op = (float *)c->n[nxt][0], *om = (float *)c->n[nxt][1];
    const Zm2Conf &z = c->zm2;
    const bool per = c->p.lateral_bc == IT_PERIODIC;
    const int nw = z.threads / 32;
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    const bool sc = c->p.space_charge != 0;
#define ZM2_LAUNCH(P, W, S)                                                                              \
    if (per == P && nw == W && sc == S)                                                                  \
        step_zmarch2_kernel<P, W, S><<<z.grid, W * 32, z.smem, s>>>(maps, op, om, nx, ny, nz, z, c->cf, c->d_slots, \
                                                                   c->d_err);
    ZM2_LAUNCH(true, 16, false) ZM2_LAUNCH(true, 8, false) ZM2_LAUNCH(false, 16, false) ZM2_LAUNCH(false, 8, false)
    ZM2_LAUNCH(true, 16, true) ZM2_LAUNCH(true, 8, true) ZM2_LAUNCH(false, 16, true) ZM2_LAUNCH(false, 8, true)
#undef ZM2_LAUNCH
    IT_CK(cudaGetLastError());
    c->cur = nxt;
    return IT_OK;
}

}  // namespace itk
