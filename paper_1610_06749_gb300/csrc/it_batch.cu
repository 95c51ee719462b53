// it_batch.cu -- many independent simulations advanced by one launch per step.
//
// Each simulation is the same method as a single context (Eq. theEquation
// discretised as in the Appendix, deposition of Eqs. linear_density /
// Gaussian / created, electrode tallies and f of Eq. collection_efficiency)
// on its own grid, dx, voltage and time step.  All simulations live in four
// shared FP32 arrays (two ping-pong sets of n+ and n-), each simulation
// aligned to 256 bytes.  A work table lists (simulation, row range) entries;
// one launch of step_batched_kernel advances every active simulation by one
// of its own steps, and segments of launches are replayed from a CUDA graph.
// At segment ends the per-entry tally slots are folded into per-simulation
// FP64 accumulators in a fixed order, in-domain charge is measured, and
// finished simulations leave the table.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "it_device.cuh"
#include "it_internal.cuh"
#include "it_tma.cuh"

namespace itk {

struct BatchSim {
    int nx, ny, nz, pad;
    long long off;          // element offset of this simulation in each state array
    Coef<float> cf;
};

struct BatchEntry {
    int sim, pad;
    long long begin, end;   // row range inside the simulation (row = k * ny + j)
};

// One explicit step of the rows [begin, end) of one simulation; the same
// per-cell operation sequence as the single-simulation kernels.  Thread t
// owns x = t mod nx of every (256 / nx)-th row, so there is no division per
// cell.
template <bool PERIODIC, bool SC>
__global__ void __launch_bounds__(256)
step_batched_kernel(const BatchSim *__restrict__ sims, const BatchEntry *__restrict__ tab,
                    const float *__restrict__ ip_all, const float *__restrict__ im_all, float *__restrict__ op_all,
                    float *__restrict__ om_all, double *__restrict__ slots) {
    constexpr int NQ = SC ? 9 : 7;   // tallies: 7, 9 with space charge
    __shared__ double red[32 * NQ];
    __shared__ BatchSim S;
    __shared__ BatchEntry E;
    if (threadIdx.x == 0) {
        E = tab[blockIdx.x];
        S = sims[E.sim];
    }
    __syncthreads();
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const Coef<float> &c = S.cf;
    const float *ip = ip_all + S.off, *im = im_all + S.off;
    float *op = op_all + S.off, *om = om_all + S.off;
    const int plane = nx * ny;
    const int R = nx <= (int)blockDim.x ? (int)blockDim.x / nx : 1;   // rows per pass
    const int lane_row = nx <= (int)blockDim.x ? (int)threadIdx.x / nx : 0;
    double acc[NQ] = {};
    if (lane_row < R) {
        const int i0 = nx <= (int)blockDim.x ? (int)threadIdx.x - lane_row * nx : (int)threadIdx.x;
        long long row = E.begin + lane_row;
        int k = (int)(row / ny), j = (int)(row - (long long)k * ny);
        for (; row < E.end; row += R) {
            for (int i = i0; i < nx; i += (nx <= (int)blockDim.x ? nx : (int)blockDim.x)) {
                const int idx = (k * ny + j) * nx + i;
                const int ixm = (i > 0) ? idx - 1 : idx + (nx - 1);
                const int ixp = (i < nx - 1) ? idx + 1 : idx - (nx - 1);
                const int iym = (j > 0) ? idx - nx : idx + (ny - 1) * nx;
                const int iyp = (j < ny - 1) ? idx + nx : idx - (ny - 1) * nx;
                const float p0 = ip[idx], m0 = im[idx];
                const float rr = p0 * m0;
                acc[0] += (double)rr;
                const int cx = (i == 0) + (i == nx - 1);
                const int cy = (j == 0) + (j == ny - 1);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float *in = s ? im : ip;
                    const float n0 = s ? m0 : p0;
                    const float xm = (PERIODIC || i > 0) ? in[ixm] : 0.f;
                    const float xp = (PERIODIC || i < nx - 1) ? in[ixp] : 0.f;
                    const float ym = (PERIODIC || j > 0) ? in[iym] : 0.f;
                    const float yp = (PERIODIC || j < ny - 1) ? in[iyp] : 0.f;
                    const float zm = (k > 0) ? in[idx - plane] : 0.f;
                    const float zp = (k < nz - 1) ? in[idx + plane] : 0.f;
                    float v =
                        upd7(n0, xm, xp, ym, yp, zm, zp, rr, c.wx[s], c.wzm[s], c.wzp[s], c.adt);
                    if constexpr (SC) {
                        v = add_sc(v, c.sc[s], n0, p0, m0);
                        acc[NQ - 2 + s] += (double)__fmul_rn(n0, __fsub_rn(p0, m0));
                    }
                    (s ? om : op)[idx] = v;
                    if (k == 0) acc[1 + s] += (double)n0;
                    if (k == nz - 1) acc[3 + s] += (double)n0;
                    if (!PERIODIC && (cx | cy)) acc[5 + s] += (double)n0 * (cx * c.latx_f[s] + cy * c.laty_f[s]);
                }
            }
            j += R;
            while (j >= ny) { j -= ny; ++k; }
        }
    }
    block_sum<NQ>(acc, red);
    if (threadIdx.x == 0) {
        double *sl = slots + (size_t)blockIdx.x * NT;
        sl[0] += acc[0] * c.rec_f;
        sl[1] += acc[1] * c.anode_f[0];
        sl[2] += acc[2] * c.anode_f[1];
        sl[3] += acc[3] * c.cathode_f[0];
        sl[4] += acc[4] * c.cathode_f[1];
        sl[5] += acc[5];
        sl[6] += acc[6];
        if constexpr (SC) {
            sl[7] += acc[NQ - 2] * c.sc_f[0];
            sl[8] += acc[NQ - 1] * c.sc_f[1];
        }
    }
}

// Entry of the float4 kernel: rows [y0, y0 + rows) of one simulation,
// planes [z0, z1).
struct VecEntry {
    int sim, y0, rows, z0, z1, pad;
};

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// Float4 z-march for simulations with nx % 4 == 0: thread t owns x-segment
// 4 (t mod nx/4) of row t div (nx/4), keeps planes k-1, k, k+1 of it in
// registers, reads the y-neighbour rows with 16-byte loads (mostly L1/L2
// hits: they are other threads' centres), and takes x-neighbours by warp
// shuffle.  Same per-cell operation sequence as every other kernel.
template <bool PERIODIC, bool SC>
__global__ void __launch_bounds__(256, 3)
step_batched_vec_kernel(const BatchSim *__restrict__ sims, const VecEntry *__restrict__ tab,
                        const float *__restrict__ ip_all, const float *__restrict__ im_all,
                        float *__restrict__ op_all, float *__restrict__ om_all, double *__restrict__ slots) {
    // per-warp FP64 tallies (tally q of warp w at w*WQ+q): 7 tallies, 9 with
    // space charge; a power-of-two row keeps the index a shift
    constexpr int WQ = SC ? 16 : 8, NQ = SC ? 9 : 7;
    __shared__ double wacc[8 * WQ];
    __shared__ BatchSim S;
    __shared__ VecEntry E;
    if (threadIdx.x == 0) {
        E = tab[blockIdx.x];
        S = sims[E.sim];
    }
    if (threadIdx.x < 8 * WQ) wacc[threadIdx.x] = 0.0;
    __syncthreads();
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const Coef<float> &c = S.cf;
    const float *in_[2] = {ip_all + S.off, im_all + S.off};
    float *out_[2] = {op_all + S.off, om_all + S.off};
    const int plane = nx * ny;
    const int ncol4 = nx >> 2;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int ty = t / ncol4, c4 = t - (t / ncol4) * ncol4;
    const bool valid = ty < E.rows;
    const int yg = E.y0 + (valid ? ty : E.rows - 1);
    const int x0 = 4 * c4;
    const int row = yg * nx + x0;
    const bool edge_u = yg == 0, edge_d = yg == ny - 1;
    const int row_u = (edge_u ? ny - 1 : yg - 1) * nx + x0;
    const int row_d = (edge_d ? 0 : yg + 1) * nx + x0;
    const bool zero_u = !PERIODIC && edge_u, zero_d = !PERIODIC && edge_d;
    const bool need_l = lane == 0 || c4 == 0, need_r = lane == 31 || c4 == ncol4 - 1;
    const int row_l = yg * nx + (c4 == 0 ? nx - 1 : x0 - 1);
    const int row_r = yg * nx + (c4 == ncol4 - 1 ? 0 : x0 + 4);
    const bool zero_l = !PERIODIC && c4 == 0, zero_r = !PERIODIC && c4 == ncol4 - 1;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // warp-uniform: one FP32 partial per lane, reduced in FP64 (fixed order)
    // into the warp's tally q
    auto flush = [&](int q, float part) {
        double v = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wacc[warp * WQ + q] += v;
    };
    float4 prev[2], cur[2], nxt[2];
    for (int s = 0; s < 2; ++s) {
        prev[s] = E.z0 > 0 ? ldg4(in_[s] + (E.z0 - 1) * plane + row) : zero4;
        cur[s] = ldg4(in_[s] + E.z0 * plane + row);
        nxt[s] = E.z0 + 1 < nz ? ldg4(in_[s] + (E.z0 + 1) * plane + row) : zero4;
    }
    float rsum = 0.f, lsum0 = 0.f, lsum1 = 0.f, ssum0 = 0.f, ssum1 = 0.f;
    int nacc = 0;
    for (int k = E.z0; k < E.z1; ++k) {
        const int pk = k * plane;
        float4 nn[2];   // two planes ahead: more loads in flight per thread
#pragma unroll
        for (int s = 0; s < 2; ++s) nn[s] = k + 2 < nz ? ldg4(in_[s] + pk + 2 * plane + row) : zero4;
        const float2 rxy = __fmul2_rn(make_float2(cur[0].x, cur[0].y), make_float2(cur[1].x, cur[1].y));
        const float2 rzw = __fmul2_rn(make_float2(cur[0].z, cur[0].w), make_float2(cur[1].z, cur[1].w));
        float an[2] = {0.f, 0.f}, lat[2] = {0.f, 0.f};
        float2 dxy, dzw;
        if (SC) sc_diff4(cur[0], cur[1], dxy, dzw);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float4 n = cur[s];
            const float4 u = zero_u ? zero4 : ldg4(in_[s] + pk + row_u);
            const float4 d = zero_d ? zero4 : ldg4(in_[s] + pk + row_d);
            float l = __shfl_up_sync(0xffffffffu, n.w, 1);
            float r = __shfl_down_sync(0xffffffffu, n.x, 1);
            if (need_l) l = zero_l ? 0.f : __ldg(in_[s] + pk + row_l);
            if (need_r) r = zero_r ? 0.f : __ldg(in_[s] + pk + row_r);
            float4 v = upd7x4(n, l, r, u, d, prev[s], nxt[s], rxy, rzw, c.wx[s], c.wzm[s],
                              c.wzp[s], c.adt);
            if (SC) {
                float2 pxy, pzw;
                v = add_sc4(v, c.sc[s], n, dxy, dzw, pxy, pzw);
                if (valid) (s ? ssum1 : ssum0) += (pxy.x + pxy.y) + (pzw.x + pzw.y);
            }
            if (valid) {
                *reinterpret_cast<float4 *>(out_[s] + pk + row) = v;
                if (k == 0 || k == nz - 1) an[s] += (n.x + n.y) + (n.z + n.w);
                if (!PERIODIC) {
                    if (c4 == 0) lat[s] += n.x;
                    if (c4 == ncol4 - 1) lat[s] += n.w;
                    if (edge_u) lat[s] += (n.x + n.y) + (n.z + n.w);
                    if (edge_d) lat[s] += (n.x + n.y) + (n.z + n.w);
                }
            }
            prev[s] = n;
            cur[s] = nxt[s];
            nxt[s] = nn[s];
        }
        if (valid) rsum += (rxy.x + rxy.y) + (rzw.x + rzw.y);
        if (!PERIODIC) { lsum0 += lat[0]; lsum1 += lat[1]; }
        // FP32 partials over at most 32 planes, then FP64
        if (++nacc == 32) {
            flush(0, rsum);
            rsum = 0.f;
            if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); lsum0 = lsum1 = 0.f; }
            if (SC) { flush(7, ssum0); flush(8, ssum1); ssum0 = ssum1 = 0.f; }
            nacc = 0;
        }
        if (k == 0) { flush(1, an[0]); flush(2, an[1]); }
        if (k == nz - 1) { flush(3, an[0]); flush(4, an[1]); }
    }
    flush(0, rsum);
    if (!PERIODIC) { flush(5, lsum0); flush(6, lsum1); }
    if (SC) { flush(7, ssum0); flush(8, ssum1); }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc[NQ];
        for (int q = 0; q < NQ; ++q) {
            double v = 0.0;
            for (int w = 0; w < 8; ++w) v += wacc[w * WQ + q];
            acc[q] = v;
        }
        double *sl = slots + (size_t)blockIdx.x * NT;
        sl[0] += acc[0] * c.rec_f;
        sl[1] += acc[1] * c.anode_f[0];
        sl[2] += acc[2] * c.anode_f[1];
        sl[3] += acc[3] * c.cathode_f[0];
        sl[4] += acc[4] * c.cathode_f[1];
        // lateral faces: x and y weights are equal for dx = dy (latx_f == laty_f)
        sl[5] += acc[5] * c.latx_f[0];
        sl[6] += acc[6] * c.latx_f[1];
        if (SC) {
            sl[7] += acc[NQ - 2] * c.sc_f[0];
            sl[8] += acc[NQ - 1] * c.sc_f[1];
        }
    }
}

// TMA-staged float4 z-march over the entries of simulations with nx % 4 == 0
// and nx <= 256: the batched counterpart of the single-context step kernel.
// A CTA owns rows [y0, y0 + rows) of one simulation (full width) and planes
// [z0, z1).  Every plane it needs (z0 - 1 .. z1) arrives by TMA in a ring of
// shared-memory slots: a box of bt = min(256 IPT / (nx/4), 256, ny) rows per
// species plus one halo row above and below, wrapped when the faces are
// periodic; rows and planes outside the simulation's tensor arrive as zeros
// (the absorbing faces and the electrode ghost planes).  Each simulation's
// tensor maps (two sets x two species x {main box for IPT = 1, main box for
// IPT = 2, halo row}) sit in global memory.  The last warp to release a slot
// refills it with the plane S further on.  Thread t owns the IPT float4
// x-segments q = t + 256 it (segment q mod (nx/4) of row q div (nx/4)),
// keeps planes k-1 and k of them in registers and reads x/y neighbours and
// plane k+1 from shared memory: the same per-cell operation sequence as
// every other kernel.  IPT = 1 runs three CTAs per SM, IPT = 2 two with
// larger rings; a plane's round through the CTA sets the time, and two
// float4 per thread halve the rounds per cell.  Every ring wait is bounded
// (2^32 SM cycles); a wait that runs out raises the error flag, and the CTA
// drains the copies it issued and returns.
constexpr int BT_MAX_S = 8;
constexpr int BT_WARPS = 8;
// dynamic shared memory of the TMA batched kernel with one float4 per thread:
// three CTAs per SM; the ring gets whatever slots fit (3..8; a slot is at
// most 12 KiB at nx = 256)
constexpr int kBtSmem = 70 * 1024;
constexpr int kBtSmemFloats = (kBtSmem - 128) / 4;
// with two float4 per thread: two CTAs per SM, twice the rows per box
constexpr int kBtSmem2 = 105 * 1024;
constexpr int kBtSmemFloats2 = (kBtSmem2 - 128) / 4;
// tensor maps per simulation: [set][species][main box of one float4 per
// thread, main box of two, halo row]
constexpr int BT_MAPS = 12;

__device__ __forceinline__ int bt_align32(int f) { return (f + 31) & ~31; }

template <bool PERIODIC, bool SC, int IPT>
__global__ void __launch_bounds__(BT_WARPS * 32, (IPT == 1 ? 3 : 2))
step_batched_tma_kernel(const BatchSim *__restrict__ sims, const VecEntry *__restrict__ tab,
                        const CUtensorMap *__restrict__ maps, int parity, float *__restrict__ op_all,
                        float *__restrict__ om_all, double *__restrict__ slots, int smem_floats,
                        int *__restrict__ err) {
    constexpr int NW = BT_WARPS, WQ = SC ? 16 : 8, NQ = SC ? 9 : 7;
    extern __shared__ __align__(128) unsigned char bt_smem_raw[];
    unsigned char *smem_base = bt_smem_raw + ((128u - (smem_u32(bt_smem_raw) & 127u)) & 127u);
    float *ring = reinterpret_cast<float *>(smem_base);
    __shared__ double wacc[NW * WQ];
    __shared__ __align__(8) uint64_t full[BT_MAX_S];
    __shared__ uint32_t rel[BT_MAX_S], fills[BT_MAX_S];
    __shared__ volatile int abort_flag;
    __shared__ BatchSim Sm;
    __shared__ VecEntry E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        E = tab[blockIdx.x];
        Sm = sims[E.sim];
    }
    __syncthreads();
    const int nx = Sm.nx, ny = Sm.ny, nz = Sm.nz;
    const Coef<float> &c = Sm.cf;
    // the weights in registers for the march (read from shared memory at
    // every plane otherwise)
    const float rwx[2] = {c.wx[0], c.wx[1]}, rwzm[2] = {c.wzm[0], c.wzm[1]}, rwzp[2] = {c.wzp[0], c.wzp[1]};
    const float radt = c.adt;
    const int ncol4 = nx >> 2;
    const int bt = min(min(256 * IPT / ncol4, 256), ny);   // rows of the main box (a box dimension is <= 256)
    const int rows = E.rows;                        // rows computed (<= bt)
    const int reg_main = bt_align32(nx), reg_bot = reg_main + bt_align32(bt * nx), blk = reg_bot + bt_align32(nx);
    const int slotf = 2 * blk;
    const int S = min(smem_floats / slotf, BT_MAX_S);   // the host keeps this >= 3
    const CUtensorMap *mp = maps + (size_t)E.sim * BT_MAPS + parity * 6;   // [species][main1, main2, halo]
    const int z0 = E.z0, z1 = E.z1, y0 = E.y0;
    const int nload = z1 - z0 + 2;                  // planes z0 - 1 .. z1
    const int ytop = PERIODIC ? (y0 > 0 ? y0 - 1 : ny - 1) : y0 - 1;
    const int ybot = PERIODIC ? (y0 + rows < ny ? y0 + rows : 0) : y0 + rows;
    const uint32_t tx = 2u * (uint32_t)(bt + 2) * (uint32_t)nx * 4u;

    // load plane z0 - 1 + n into its slot (one thread)
    auto issue = [&](int n) {
        const int p = z0 - 1 + n;
        const int slot = n % S;
        float *base = ring + (size_t)slot * slotf;
        uint64_t *bar = &full[slot];
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, tx);
        for (int s = 0; s < 2; ++s) {
            float *b = base + s * blk;
            tma_load3(b + reg_main, &mp[3 * s + IPT - 1], bar, 0, y0, p);
            tma_load3(b, &mp[3 * s + 2], bar, 0, ytop, p);
            tma_load3(b + reg_bot, &mp[3 * s + 2], bar, 0, ybot, p);
        }
        fills[slot] += 1;
    };

    if (tid == 0) {
        for (int q = 0; q < 6; ++q) fence_tensormap_acquire(&mp[q]);
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            rel[q] = 0;
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

    // this thread's float4 segments q = tid + 256 it; threads past the tile
    // repeat its last segment and store nothing
    bool valid[IPT], edge_u[IPT], edge_d[IPT];
    int c4_[IPT], o_c[IPT], o_u[IPT], o_d[IPT], o_l[IPT], o_r[IPT];
    uint32_t off[IPT];
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int q = tid + it * BT_WARPS * 32;
        valid[it] = q < rows * ncol4;
        const int te = valid[it] ? q : rows * ncol4 - 1;
        const int ty = te / ncol4, c4 = te - ty * ncol4;
        const int x0 = 4 * c4;
        c4_[it] = c4;
        o_c[it] = reg_main + ty * nx + x0;
        o_u[it] = ty == 0 ? x0 : reg_main + (ty - 1) * nx + x0;
        o_d[it] = ty == rows - 1 ? reg_bot + x0 : reg_main + (ty + 1) * nx + x0;
        o_l[it] = reg_main + ty * nx + (c4 == 0 ? nx - 1 : x0 - 1);
        o_r[it] = reg_main + ty * nx + (c4 == ncol4 - 1 ? 0 : x0 + 4);
        const int yg = y0 + ty;
        edge_u[it] = !PERIODIC && yg == 0;
        edge_d[it] = !PERIODIC && yg == ny - 1;
        off[it] = ((uint32_t)z0 * (uint32_t)ny + (uint32_t)yg) * (uint32_t)nx + (uint32_t)x0;
    }
    float *out_[2] = {op_all + Sm.off, om_all + Sm.off};

    RingPos pos{0, 0u};
    int nrel = 0;
    bool failed = false;
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
    auto release = [&](const RingPos &u) {
        __syncwarp();
        if (lane == 0 && !failed) {
            const uint32_t old = atom_add_acq_rel(&rel[u.slot], 1u);
            if (old % NW == NW - 1 && nrel + S < nload && !abort_flag) issue(nrel + S);
        }
        ++nrel;
    };

    float4 prev[IPT][2], cur[IPT][2];
    wait_full(pos);
    {
        const float *sl = ring + (size_t)pos.slot * slotf;
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            prev[it][0] = *reinterpret_cast<const float4 *>(sl + o_c[it]);
            prev[it][1] = *reinterpret_cast<const float4 *>(sl + blk + o_c[it]);
        }
    }
    release(pos);
    pos.advance(S);
    wait_full(pos);
    RingPos pc = pos;
    pos.advance(S);
    {
        const float *sl = ring + (size_t)pc.slot * slotf;
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            cur[it][0] = *reinterpret_cast<const float4 *>(sl + o_c[it]);
            cur[it][1] = *reinterpret_cast<const float4 *>(sl + blk + o_c[it]);
        }
    }
    float rsum = 0.f, lsum0 = 0.f, lsum1 = 0.f, ssum0 = 0.f, ssum1 = 0.f;
    int nacc = 0;
    for (int k = z0; k < z1; ++k) {
        wait_full(pos);
        const float *sk = ring + (size_t)pc.slot * slotf;
        const float *sn = ring + (size_t)pos.slot * slotf;
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
                const float *bk = sk + s * blk;
                const float4 n = cur[it][s];
                const float4 u = *reinterpret_cast<const float4 *>(bk + o_u[it]);
                const float4 d = *reinterpret_cast<const float4 *>(bk + o_d[it]);
                const float4 zp = *reinterpret_cast<const float4 *>(sn + s * blk + o_c[it]);
                float l = bk[o_l[it]];
                float r = bk[o_r[it]];
                if (!PERIODIC) {
                    if (c4_[it] == 0) l = 0.f;
                    if (c4_[it] == ncol4 - 1) r = 0.f;
                }
                float4 v = upd7x4(n, l, r, u, d, prev[it][s], zp, rxy, rzw, rwx[s], rwzm[s], rwzp[s], radt);
                if (SC) {
                    float2 pxy, pzw;
                    v = add_sc4(v, c.sc[s], n, dxy, dzw, pxy, pzw);
                    if (valid[it]) (s ? ssum1 : ssum0) += (pxy.x + pxy.y) + (pzw.x + pzw.y);
                }
                if (valid[it]) {
                    *reinterpret_cast<float4 *>(out_[s] + off[it]) = v;
                    if (k == 0 || k == nz - 1) an[s] += (n.x + n.y) + (n.z + n.w);
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
    release(pc);   // plane z1
    if (failed && lane == 0) atomicExch(err, 1);
    __syncthreads();
    if (tid == 0) {
        // no copy may be in flight when the CTA exits
        for (int j = 0; j < S; ++j)
            if (fills[j] > 0) (void)mbar_wait_bounded(&full[j], (fills[j] - 1u) & 1u);
    }
    if (tid == 0 && !abort_flag) {
        double acc[NQ];
        for (int q = 0; q < NQ; ++q) {
            double v = 0.0;
            for (int w = 0; w < NW; ++w) v += wacc[w * WQ + q];
            acc[q] = v;
        }
        double *sl = slots + (size_t)blockIdx.x * NT;
        sl[0] += acc[0] * c.rec_f;
        sl[1] += acc[1] * c.anode_f[0];
        sl[2] += acc[2] * c.anode_f[1];
        sl[3] += acc[3] * c.cathode_f[0];
        sl[4] += acc[4] * c.cathode_f[1];
        sl[5] += acc[5] * c.latx_f[0];
        sl[6] += acc[6] * c.latx_f[1];
        if (SC) {
            sl[7] += acc[NQ - 2] * c.sc_f[0];
            sl[8] += acc[NQ - 1] * c.sc_f[1];
        }
    }
}

// Fold the slots of each active simulation's entries (contiguous in the
// table, in order) into its FP64 accumulators and clear them.  One block
// per active simulation, one thread per tally.
__global__ void batch_fold_kernel(const int *__restrict__ first, const int *__restrict__ count,
                                  const int *__restrict__ sim_of, double *__restrict__ slots,
                                  double *__restrict__ acc) {
    const int a = blockIdx.x, q = threadIdx.x;
    if (q >= NT) return;
    double s = 0.0;
    for (int e = first[a]; e < first[a] + count[a]; ++e) {
        s += slots[(size_t)e * NT + q];
        slots[(size_t)e * NT + q] = 0.0;
    }
    acc[(size_t)sim_of[a] * NT + q] += s;
}

// Per-entry sums of n+ and n- for the in-domain charge: FP32 partials over
// at most 32 cells per thread, then FP64 (once per 32 cells, outside the
// per-cell loop: FP64 arithmetic is slow on this GPU).
__global__ void __launch_bounds__(256)
batch_monitor_kernel(const BatchSim *__restrict__ sims, const BatchEntry *__restrict__ tab,
                     const float *__restrict__ ip_all, const float *__restrict__ im_all, double *__restrict__ mon) {
    __shared__ double red[32 * 2];
    const BatchEntry E = tab[blockIdx.x];
    const long long off = sims[E.sim].off;
    const long long nxs = sims[E.sim].nx;
    double v[2] = {0.0, 0.0};
    const size_t end = (size_t)(E.end * nxs);
    size_t idx = (size_t)(E.begin * nxs) + threadIdx.x;
    while (idx < end) {
        float a = 0.f, b = 0.f;
        for (int j = 0; j < 32 && idx < end; ++j, idx += blockDim.x) {
            a += ip_all[off + idx];
            b += im_all[off + idx];
        }
        v[0] += (double)a;
        v[1] += (double)b;
    }
    block_sum<2>(v, red);
    if (threadIdx.x == 0) {
        mon[2 * blockIdx.x] = v[0];
        mon[2 * blockIdx.x + 1] = v[1];
    }
}

// Per-entry maximum of n+ and n-.
__global__ void __launch_bounds__(256)
batch_max_kernel(const BatchSim *__restrict__ sims, const BatchEntry *__restrict__ tab,
                 const float *__restrict__ ip_all, const float *__restrict__ im_all, float *__restrict__ mx) {
    __shared__ float red[32];
    const BatchEntry E = tab[blockIdx.x];
    const long long off = sims[E.sim].off;
    const long long nxs = sims[E.sim].nx;
    float v = -INFINITY;
    for (size_t idx = (size_t)(E.begin * nxs) + threadIdx.x; idx < (size_t)(E.end * nxs); idx += blockDim.x)
        v = fmaxf(v, fmaxf(ip_all[off + idx], im_all[off + idx]));
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
        mx[blockIdx.x] = v;
    }
}

}  // namespace itk

using namespace itk;

struct it_batch {
    int nsim;
    it_params p;
    std::vector<it_sim_desc> desc;
    std::vector<BatchSim> hs;         // host copy of the descriptors
    std::vector<double> dx;
    std::vector<double> dt;
    size_t total;                     // elements per state array
    float *state[2][2];               // [set][species]
    void *state_base;
    BatchSim *d_sims;
    double *d_acc;                    // [nsim][NT] folded tallies
    double *d_rel;                    // [nsim][8] released (DevAcc layout)
    // work tables of the current segment
    std::vector<BatchEntry> tab;      // row ranges of every active simulation (monitors)
    std::vector<int> mfirst, mcount;  // per active simulation, into tab
    std::vector<int> morder;          // the active simulation of each mfirst/mcount entry
    std::vector<VecEntry> vtab;       // step entries of the float4 kernel
    std::vector<BatchEntry> stab;     // step entries of the scalar kernel
    std::vector<int> first, count, sim_of;   // per active simulation, into the step slots
    BatchEntry *d_tab, *d_stab;
    VecEntry *d_vtab;
    int *d_first, *d_count, *d_simof;
    double *d_slots, *d_mon;
    float *d_max;                     // per-entry peak density (the dt ladder)
    size_t tab_cap, stab_cap, vtab_cap, slot_cap, act_cap, max_cap;
    long long chunk;                  // cells per entry
    int vec_cps;                      // CTAs per SM the float4 launch aims for (sets its z split)
    // per simulation
    std::vector<int64_t> steps;
    std::vector<double> t_s;          // simulated time: the sum of every step's dt
    std::vector<char> active;
    int64_t bstep;                    // steps taken by every active simulation
    cudaStream_t stream;
    cudaGraphExec_t graph;
    int graph_len, graph_parity;
    bool tab_dirty;
    // pulse trains: each simulation's deposited tracks are re-deposited every
    // period_steps steps until count pulses have been released
    std::vector<std::vector<double>> pulse_tracks;   // packed [n][4]
    std::vector<int32_t> pulse_count, pulse_done;
    std::vector<int64_t> pulse_period;
    // deposition scratch (sized for the largest simulation)
    double *d_plane, *d_tracks, *d_wx, *d_wy;
    int64_t track_cap;
    int max_nx, max_ny;
    // TMA-staged float4 kernel: per simulation [set][species][main, halo]
    // tensor maps (zero for simulations it does not take), its use, the
    // number of leading float4 entries it runs, and the device error flag of
    // its bounded waits
    CUtensorMap *d_maps;
    std::vector<char> tma_ok;
    int use_tma;
    int tma_ipt;                      // float4 per thread of the TMA kernel (1 or 2)
    int nvt;
    int *d_err;
};

namespace {

int bfail(int code, const std::string &m) {
    set_error(m);
    return code;
}

// Rebuild the work tables for the active simulations.  Step entries: the
// float4 kernel takes simulations with nx % 4 == 0 (tiles of 256/(nx/4)
// rows, split in z when few cells are active), the scalar kernel the rest.
// All entries of one simulation are contiguous, so the fold is in order.
int build_table(it_batch *b) {
    b->tab.clear(); b->mfirst.clear(); b->mcount.clear(); b->morder.clear();
    b->vtab.clear(); b->stab.clear();
    b->first.clear(); b->count.clear(); b->sim_of.clear();
    long long active_cells = 0, vec_tiles = 0;
    for (int s = 0; s < b->nsim; ++s) {
        if (!b->active[s]) continue;
        const BatchSim &h = b->hs[s];
        active_cells += (long long)h.nx * h.ny * h.nz;
        if (h.nx % 4 == 0 && h.nx <= 1024) {
            const int rows = std::max(1, 256 / (h.nx / 4));
            vec_tiles += (h.ny + rows - 1) / rows;
        }
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long chunk = std::max(1024LL, std::min(b->chunk, active_cells / (4LL * sms)));
    // z splits so that the float4 launch keeps about vec_cps CTAs per SM busy
    const long long zsplit =
        vec_tiles > 0 ? std::max(1LL, ((long long)b->vec_cps * sms + vec_tiles - 1) / vec_tiles) : 1;
    std::vector<int> vfirst, vcount, sfirst, scount, vsim, ssim;
    // float4 entries of the simulations the TMA kernel takes come first
    b->nvt = 0;
    std::vector<int> order;
    for (int pass = 0; pass < 2; ++pass)
        for (int s = 0; s < b->nsim; ++s)
            if (b->active[s] && ((b->use_tma && b->tma_ok[s]) == (pass == 0))) order.push_back(s);
    for (int s : order) {
        const BatchSim &h = b->hs[s];
        const long long rows = (long long)h.ny * h.nz;
        const long long rpe = std::max(1LL, chunk / h.nx);
        b->mfirst.push_back((int)b->tab.size());
        int n = 0;
        for (long long r0 = 0; r0 < rows; r0 += rpe, ++n) b->tab.push_back(BatchEntry{s, 0, r0, std::min(rows, r0 + rpe)});
        b->mcount.push_back(n);
        b->morder.push_back(s);
        if (h.nx % 4 == 0 && h.nx <= 1024) {
            // rows per entry: a 256-thread tile of float4 (times the TMA
            // kernel's float4 per thread for the simulations it takes)
            const int ipt = (b->use_tma && b->tma_ok[s]) ? b->tma_ipt : 1;
            const int rpt = std::max(1, std::min(256 * ipt / (h.nx / 4), 256));
            const int zc = (int)std::min<long long>(zsplit, std::max(1, h.nz / 8));
            vsim.push_back(s);
            vfirst.push_back((int)b->vtab.size());
            int m = 0;
            for (int y0 = 0; y0 < h.ny; y0 += rpt)
                for (int q = 0; q < zc; ++q, ++m)
                    b->vtab.push_back(VecEntry{s, y0, std::min(rpt, h.ny - y0), (int)((long long)h.nz * q / zc),
                                               (int)((long long)h.nz * (q + 1) / zc), 0});
            vcount.push_back(m);
            if (b->use_tma && b->tma_ok[s]) b->nvt += m;
        } else {
            ssim.push_back(s);
            sfirst.push_back((int)b->stab.size());
            int m = 0;
            for (long long r0 = 0; r0 < rows; r0 += rpe, ++m) b->stab.push_back(BatchEntry{s, 0, r0, std::min(rows, r0 + rpe)});
            scount.push_back(m);
        }
    }
    // step slots: [float4 entries][scalar entries]
    const int nv = (int)b->vtab.size();
    for (size_t q = 0; q < vsim.size(); ++q) { b->sim_of.push_back(vsim[q]); b->first.push_back(vfirst[q]); b->count.push_back(vcount[q]); }
    for (size_t q = 0; q < ssim.size(); ++q) { b->sim_of.push_back(ssim[q]); b->first.push_back(nv + sfirst[q]); b->count.push_back(scount[q]); }
    const size_t ne = b->tab.size(), nvs = b->vtab.size(), nss = b->stab.size(), na = b->sim_of.size();
    const size_t nslot = nvs + nss;
    auto grow = [&](void **p, size_t &cap, size_t need, size_t esz) -> cudaError_t {
        if (need <= cap) return cudaSuccess;
        cudaFree(*p);
        *p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(p, esz * need);
        if (e == cudaSuccess) cap = need;
        return e;
    };
    size_t mon_cap = b->tab_cap;
    IT_CK(grow((void **)&b->d_tab, b->tab_cap, ne, sizeof(BatchEntry)));
    if (b->tab_cap != mon_cap || !b->d_mon) {
        cudaFree(b->d_mon);
        b->d_mon = nullptr;
        IT_CK(cudaMalloc(&b->d_mon, sizeof(double) * 2 * std::max<size_t>(b->tab_cap, 1)));
    }
    IT_CK(grow((void **)&b->d_vtab, b->vtab_cap, nvs, sizeof(VecEntry)));
    IT_CK(grow((void **)&b->d_stab, b->stab_cap, nss, sizeof(BatchEntry)));
    IT_CK(grow((void **)&b->d_slots, b->slot_cap, nslot, sizeof(double) * NT));
    if (na > b->act_cap) {
        cudaFree(b->d_first); cudaFree(b->d_count); cudaFree(b->d_simof);
        IT_CK(cudaMalloc(&b->d_first, sizeof(int) * na));
        IT_CK(cudaMalloc(&b->d_count, sizeof(int) * na));
        IT_CK(cudaMalloc(&b->d_simof, sizeof(int) * na));
        b->act_cap = na;
    }
    if (ne) IT_CK(cudaMemcpyAsync(b->d_tab, b->tab.data(), sizeof(BatchEntry) * ne, cudaMemcpyHostToDevice, b->stream));
    if (nvs) IT_CK(cudaMemcpyAsync(b->d_vtab, b->vtab.data(), sizeof(VecEntry) * nvs, cudaMemcpyHostToDevice, b->stream));
    if (nss) IT_CK(cudaMemcpyAsync(b->d_stab, b->stab.data(), sizeof(BatchEntry) * nss, cudaMemcpyHostToDevice, b->stream));
    if (nslot) IT_CK(cudaMemsetAsync(b->d_slots, 0, sizeof(double) * NT * nslot, b->stream));
    if (na) {
        IT_CK(cudaMemcpyAsync(b->d_first, b->first.data(), sizeof(int) * na, cudaMemcpyHostToDevice, b->stream));
        IT_CK(cudaMemcpyAsync(b->d_count, b->count.data(), sizeof(int) * na, cudaMemcpyHostToDevice, b->stream));
        IT_CK(cudaMemcpyAsync(b->d_simof, b->sim_of.data(), sizeof(int) * na, cudaMemcpyHostToDevice, b->stream));
    }
    IT_CK(cudaStreamSynchronize(b->stream));   // host vectors may change at the next rebuild
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    b->tab_dirty = false;
    return IT_OK;
}

int launch_batched_step(it_batch *b, int parity) {
    const int nv = (int)b->vtab.size(), ns = (int)b->stab.size(), nt = b->nvt;
    const float *ip = b->state[parity][0], *im = b->state[parity][1];
    float *op = b->state[parity ^ 1][0], *om = b->state[parity ^ 1][1];
    const bool per = b->p.lateral_bc == IT_PERIODIC;
    const bool sc = b->p.space_charge != 0;
    if (nt) {
        const bool two = b->tma_ipt == 2;
        auto *kt = two ? (per ? (sc ? step_batched_tma_kernel<true, true, 2> : step_batched_tma_kernel<true, false, 2>)
                              : (sc ? step_batched_tma_kernel<false, true, 2> : step_batched_tma_kernel<false, false, 2>))
                       : (per ? (sc ? step_batched_tma_kernel<true, true, 1> : step_batched_tma_kernel<true, false, 1>)
                              : (sc ? step_batched_tma_kernel<false, true, 1> : step_batched_tma_kernel<false, false, 1>));
        kt<<<nt, BT_WARPS * 32, two ? kBtSmem2 : kBtSmem, b->stream>>>(b->d_sims, b->d_vtab, b->d_maps, parity, op,
                                                                       om, b->d_slots,
                                                                       two ? kBtSmemFloats2 : kBtSmemFloats, b->d_err);
        IT_CK(cudaGetLastError());
    }
    if (nv > nt) {
        auto *kv = per ? (sc ? step_batched_vec_kernel<true, true> : step_batched_vec_kernel<true, false>)
                       : (sc ? step_batched_vec_kernel<false, true> : step_batched_vec_kernel<false, false>);
        kv<<<nv - nt, 256, 0, b->stream>>>(b->d_sims, b->d_vtab + nt, ip, im, op, om, b->d_slots + (size_t)NT * nt);
        IT_CK(cudaGetLastError());
    }
    if (ns) {
        double *sl = b->d_slots + (size_t)NT * nv;
        auto *ks = per ? (sc ? step_batched_kernel<true, true> : step_batched_kernel<true, false>)
                       : (sc ? step_batched_kernel<false, true> : step_batched_kernel<false, false>);
        ks<<<ns, 256, 0, b->stream>>>(b->d_sims, b->d_stab, ip, im, op, om, sl);
        IT_CK(cudaGetLastError());
    }
    return IT_OK;
}

// K steps of every active simulation (K even: the graph returns to the same set)
int run_segment(it_batch *b, int K) {
    const int parity = (int)(b->bstep & 1);
    if (!b->graph || b->graph_len != K || b->graph_parity != parity) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaGraph_t g = nullptr;
        IT_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = IT_OK;
        for (int q = 0; q < K && rc == IT_OK; ++q) rc = launch_batched_step(b, parity ^ (q & 1));
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(batch)");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate(batch)"); }
        b->graph_len = K;
        b->graph_parity = parity;
    }
    IT_CK(cudaGraphLaunch(b->graph, b->stream));
    b->bstep += K;
    for (int s = 0; s < b->nsim; ++s)
        if (b->active[s]) {
            b->steps[s] += K;
            b->t_s[s] += b->dt[s] * K;
        }
    return IT_OK;
}

// The doubling ladder of it_run_to_completion, per active simulation with no
// pulse still to come: one pass for the peak density of every table entry,
// then each simulation's dt rises to its largest admissible rung.  The step
// graph reads the descriptors from device memory, so only they change.
static int ladder_batch(it_batch *b) {
    const int ne = (int)b->tab.size();
    if (!ne) return IT_OK;
    if ((size_t)ne > b->max_cap) {
        cudaFree(b->d_max);
        b->d_max = nullptr;
        b->max_cap = 0;
        IT_CK(cudaMalloc(&b->d_max, sizeof(float) * ne));
        b->max_cap = ne;
    }
    const int parity = (int)(b->bstep & 1);
    batch_max_kernel<<<ne, 256, 0, b->stream>>>(b->d_sims, b->d_tab, b->state[parity][0], b->state[parity][1],
                                                b->d_max);
    IT_CK(cudaGetLastError());
    std::vector<float> mx(ne);
    IT_CK(cudaMemcpyAsync(mx.data(), b->d_max, sizeof(float) * ne, cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaStreamSynchronize(b->stream));
    for (size_t a = 0; a < b->morder.size(); ++a) {
        const int s = b->morder[a];
        double nmax = -INFINITY;
        for (int q = b->mfirst[a]; q < b->mfirst[a] + b->mcount[a]; ++q) nmax = std::max(nmax, (double)mx[q]);
        // as in a single context, whose check runs before the deposits of its
        // step: a check at the step of the last pulse still counts that pulse
        // as to come
        const bool last_now = b->pulse_count[s] > 1 && b->pulse_done[s] == b->pulse_count[s] &&
                              b->steps[s] == (int64_t)(b->pulse_count[s] - 1) * b->pulse_period[s];
        const bool pending = (b->pulse_done[s] >= 1 && b->pulse_done[s] < b->pulse_count[s]) || last_now;
        if (pending) continue;
        const it_sim_desc &d = b->desc[s];
        it_params p = b->p;
        p.gap_cm = d.nz * d.dx_cm;
        p.voltage_V = d.voltage_V;
        const double nd = ladder_rung(&p, d.dx_cm, b->dt[s], nmax);
        if (nd > b->dt[s]) {
            b->dt[s] = nd;
            coef_f32(&p, d.dx_cm, nd, &b->hs[s].cf);
            IT_CK(cudaMemcpyAsync(b->d_sims + s, &b->hs[s], sizeof(BatchSim), cudaMemcpyHostToDevice, b->stream));
        }
    }
    IT_CK(cudaStreamSynchronize(b->stream));
    return IT_OK;
}

int fold(it_batch *b) {
    const int na = (int)b->sim_of.size();
    if (!na) return IT_OK;
    batch_fold_kernel<<<na, 32, 0, b->stream>>>(b->d_first, b->d_count, b->d_simof, b->d_slots, b->d_acc);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// in-domain ions of every simulation in the current table
int in_domain(it_batch *b, std::vector<double> &ind2) {
    ind2.assign(2 * (size_t)b->nsim, 0.0);
    const int ne = (int)b->tab.size();
    if (!ne) return IT_OK;
    const int parity = (int)(b->bstep & 1);
    batch_monitor_kernel<<<ne, 256, 0, b->stream>>>(b->d_sims, b->d_tab, b->state[parity][0], b->state[parity][1],
                                                    b->d_mon);
    IT_CK(cudaGetLastError());
    std::vector<double> mon(2 * (size_t)ne);
    int err = 0;
    IT_CK(cudaMemcpyAsync(mon.data(), b->d_mon, sizeof(double) * 2 * ne, cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaStreamSynchronize(b->stream));
    if (err) return bfail(IT_ETIMEOUT, "a bounded device wait ran out in the batched step kernel");
    for (size_t a = 0; a < b->morder.size(); ++a) {
        const int s = b->morder[a];
        const double vol = b->dx[s] * b->dx[s] * b->dx[s];
        double p = 0, m = 0;
        for (int e = b->mfirst[a]; e < b->mfirst[a] + b->mcount[a]; ++e) { p += mon[2 * e]; m += mon[2 * e + 1]; }
        ind2[2 * s] = p * vol;
        ind2[2 * s + 1] = m * vol;
    }
    return IT_OK;
}

void batch_free(it_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->state_base);
    cudaFree(b->d_sims); cudaFree(b->d_acc); cudaFree(b->d_rel);
    cudaFree(b->d_tab); cudaFree(b->d_slots); cudaFree(b->d_mon); cudaFree(b->d_max);
    cudaFree(b->d_vtab); cudaFree(b->d_stab);
    cudaFree(b->d_first); cudaFree(b->d_count); cudaFree(b->d_simof);
    cudaFree(b->d_plane); cudaFree(b->d_tracks); cudaFree(b->d_wx); cudaFree(b->d_wy);
    cudaFree(b->d_maps); cudaFree(b->d_err);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

int it_batch_create(int32_t nsim, const it_sim_desc *descs, const it_params *common, it_batch **out) {
    if (!out) return bfail(IT_EINVAL, "out is NULL");
    *out = nullptr;
    if (nsim < 1 || !descs || !common) return bfail(IT_EINVAL, "need at least one simulation descriptor");
    if (common->precision != IT_FP32) return bfail(IT_EINVAL, "batched simulations use FP32 densities");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bfail(IT_ECUDA, "no CUDA device available");
    it_batch *b = new (std::nothrow) it_batch();
    if (!b) return bfail(IT_ENOMEM, "host allocation failed");
    b->nsim = nsim;
    b->p = *common;
    b->desc.assign(descs, descs + nsim);
    b->hs.resize(nsim);
    b->dx.resize(nsim);
    b->dt.resize(nsim);
    b->steps.assign(nsim, 0);
    b->t_s.assign(nsim, 0.0);
    b->active.assign(nsim, 1);
    b->pulse_tracks.assign(nsim, {});
    b->pulse_count.assign(nsim, 1);
    b->pulse_done.assign(nsim, 0);
    b->pulse_period.assign(nsim, 0);
    b->chunk = 16384;
    b->vec_cps = 4;
    b->graph_parity = -1;
    size_t off = 0;
    for (int s = 0; s < nsim; ++s) {
        const it_sim_desc &d = descs[s];
        it_params p = *common;
        p.gap_cm = d.nz * d.dx_cm;
        p.voltage_V = d.voltage_V;
        p.n_peak_cm3 = d.n_peak_cm3;
        it_grid g{d.nx, d.ny, d.nz};
        double dt = d.dt_s;
        if (!(dt > 0)) {
            int rc = it_auto_dt(&p, d.dx_cm, &dt);
            if (rc) { batch_free(b); return rc; }
        }
        int rc = validate_step_args(&p, g, d.dx_cm, dt);
        if (rc) {
            std::string m = it_last_error();
            batch_free(b);
            return bfail(rc, "simulation " + std::to_string(s) + ": " + m);
        }
        if ((long long)d.nx * d.ny * d.nz > 0x7fffffffLL) {
            batch_free(b);
            return bfail(IT_EINVAL, "simulation " + std::to_string(s) + ": more than 2^31 - 1 cells");
        }
        BatchSim &h = b->hs[s];
        h.nx = d.nx; h.ny = d.ny; h.nz = d.nz; h.pad = 0;
        h.off = (long long)off;
        coef_f32(&p, d.dx_cm, dt, &h.cf);
        b->dx[s] = d.dx_cm;
        b->dt[s] = dt;
        const size_t cells = (size_t)d.nx * d.ny * d.nz;
        off += (cells + 63) / 64 * 64;   // 256-byte aligned per simulation
        b->max_nx = std::max(b->max_nx, d.nx);
        b->max_ny = std::max(b->max_ny, d.ny);
    }
    b->total = off;
    auto bail = [&](cudaError_t e, const char *what) {
        int rc = e == cudaErrorMemoryAllocation ? bfail(IT_ENOMEM, what) : cuda_fail(e, what);
        batch_free(b);
        return rc;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
    if ((e = cudaMalloc(&b->state_base, sizeof(float) * 4 * off)) != cudaSuccess) return bail(e, "batch state");
    float *base = (float *)b->state_base;
    b->state[0][0] = base; b->state[0][1] = base + off; b->state[1][0] = base + 2 * off; b->state[1][1] = base + 3 * off;
    if ((e = cudaMemsetAsync(b->state_base, 0, sizeof(float) * 4 * off, b->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMalloc(&b->d_sims, sizeof(BatchSim) * nsim)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_acc, sizeof(double) * NT * nsim)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_rel, sizeof(double) * 8 * nsim)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_plane, sizeof(double) * 2 * b->max_nx * b->max_ny)) != cudaSuccess)   // plane + tile sums
        return bail(e, "batch scratch");
    if ((e = cudaMemcpyAsync(b->d_sims, b->hs.data(), sizeof(BatchSim) * nsim, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_acc, 0, sizeof(double) * NT * nsim, b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_rel, 0, sizeof(double) * 8 * nsim, b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return bail(e, "batch setup");
    // tensor maps of the TMA batched kernel: simulations with nx % 4 == 0 and
    // nx <= 256 (one box spans the row); main boxes of min(256 / (nx/4), ny)
    // and min(512 / (nx/4), ny) rows (one or two float4 per thread) and a
    // box of one halo row
    b->tma_ok.assign(nsim, 0);
    b->use_tma = 1;
    b->tma_ipt = 1;
    {
        std::vector<CUtensorMap> maps((size_t)nsim * BT_MAPS);
        std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
        for (int s = 0; s < nsim; ++s) {
            const BatchSim &h = b->hs[s];
            if (h.nx % 4 != 0 || h.nx > 256) continue;
            int rc = IT_OK;
            for (int set = 0; set < 2 && rc == IT_OK; ++set)
                for (int sp = 0; sp < 2 && rc == IT_OK; ++sp) {
                    float *base_s = b->state[set][sp] + h.off;
                    CUtensorMap *m = &maps[(size_t)s * BT_MAPS + set * 6 + sp * 3];
                    for (int ipt = 1; ipt <= 2 && rc == IT_OK; ++ipt)
                        rc = encode_map(&m[ipt - 1], base_s, h.nx, h.ny, h.nz, h.nx,
                                        std::min(std::min(256 * ipt / (h.nx / 4), 256), h.ny));
                    if (rc == IT_OK) rc = encode_map(&m[2], base_s, h.nx, h.ny, h.nz, h.nx, 1);
                }
            if (rc) { batch_free(b); return rc; }
            b->tma_ok[s] = 1;
        }
        if ((e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * maps.size())) != cudaSuccess ||
            (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess ||
            (e = cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                                 b->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
            return bail(e, "batch tensor maps");
        for (auto *k : {step_batched_tma_kernel<true, true, 1>, step_batched_tma_kernel<true, false, 1>,
                        step_batched_tma_kernel<false, true, 1>, step_batched_tma_kernel<false, false, 1>})
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kBtSmem)) != cudaSuccess)
                return bail(e, "cudaFuncSetAttribute(batched TMA kernel)");
        for (auto *k : {step_batched_tma_kernel<true, true, 2>, step_batched_tma_kernel<true, false, 2>,
                        step_batched_tma_kernel<false, true, 2>, step_batched_tma_kernel<false, false, 2>})
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kBtSmem2)) != cudaSuccess)
                return bail(e, "cudaFuncSetAttribute(batched TMA kernel)");
    }
    b->tab_dirty = true;
    *out = b;
    return IT_OK;
}

}  // extern "C"

namespace {

// Deposit packed tracks [n][4] into simulation `sim`'s current set.
int deposit_sim(it_batch *b, int sim, const double *packed, int64_t n) {
    if (n <= 0) return IT_OK;
    const it_sim_desc &d = b->desc[sim];
    const int parity = (int)(b->steps[sim] & 1);
    // a context view of this simulation for the shared deposition kernels
    it_ctx *v = new (std::nothrow) it_ctx();
    if (!v) return bfail(IT_ENOMEM, "host allocation failed");
    v->g = Grid{d.nx, d.ny, d.nz};
    v->dx = d.dx_cm;
    v->p = b->p;
    v->prec = IT_FP32;
    v->esize = 4;
    v->cur = 0;
    v->n[0][0] = b->state[parity][0] + b->hs[sim].off;
    v->n[0][1] = b->state[parity][1] + b->hs[sim].off;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    v->nmon = 2 * sms;
    v->d_plane = b->d_plane;
    v->d_acc = b->d_rel + (size_t)8 * sim;
    int rc = IT_OK;
    if (n > b->track_cap) {
        cudaFree(b->d_tracks); cudaFree(b->d_wx); cudaFree(b->d_wy);
        b->d_tracks = b->d_wx = b->d_wy = nullptr;
        b->track_cap = 0;
        cudaError_t e;
        if ((e = cudaMalloc(&b->d_tracks, sizeof(double) * 4 * n)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_wx, sizeof(double) * b->max_nx * n)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_wy, sizeof(double) * b->max_ny * n)) != cudaSuccess) {
            delete v;
            return cuda_fail(e, "batch track scratch");
        }
        b->track_cap = n;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_tracks, packed, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "track upload");
    v->d_tracks = b->d_tracks; v->d_wx = b->d_wx; v->d_wy = b->d_wy;
    if (rc == IT_OK) rc = launch_deposit(v, n, b->stream);
    if (rc == IT_OK) {
        e = cudaStreamSynchronize(b->stream);   // packed host memory may be freed after return
        if (e != cudaSuccess) rc = cuda_fail(e, "deposit");
    }
    delete v;
    return rc;
}

}  // namespace

extern "C" {

int it_batch_deposit_tracks(it_batch *b, int32_t sim, int64_t n, const double *xy, const double *let,
                            const double *bb) {
    if (!b || sim < 0 || sim >= b->nsim) return bfail(IT_EINVAL, "bad batch or simulation index");
    if (b->bstep != 0) return bfail(IT_ESTATE, "tracks are deposited before the first step");
    if (n < 0 || (n > 0 && (!xy || !let || !bb))) return bfail(IT_EINVAL, "bad track arrays");
    if (n == 0) return IT_OK;
    for (int64_t t = 0; t < n; ++t)
        if (!std::isfinite(xy[2 * t]) || !std::isfinite(xy[2 * t + 1]) || !(let[t] >= 0) || !std::isfinite(let[t]) ||
            !(bb[t] > 0) || !std::isfinite(bb[t]))
            return bfail(IT_EINVAL, "track values must be finite with LET >= 0 and b > 0");
    std::vector<double> packed((size_t)n * 4);
    for (int64_t t = 0; t < n; ++t) {
        packed[4 * t] = xy[2 * t]; packed[4 * t + 1] = xy[2 * t + 1];
        packed[4 * t + 2] = let[t]; packed[4 * t + 3] = bb[t];
    }
    int rc = deposit_sim(b, sim, packed.data(), n);
    if (rc) return rc;
    auto &pt = b->pulse_tracks[sim];
    pt.insert(pt.end(), packed.begin(), packed.end());
    b->pulse_done[sim] = 1;
    return IT_OK;
}

int it_batch_set_pulses(it_batch *b, int32_t sim, int32_t count, int64_t period_steps) {
    if (!b || sim < 0 || sim >= b->nsim) return bfail(IT_EINVAL, "bad batch or simulation index");
    if (b->bstep != 0) return bfail(IT_ESTATE, "pulse trains are set before the first step");
    if (count < 1 || (count > 1 && period_steps < 1)) return bfail(IT_EINVAL, "need count >= 1 and period_steps >= 1");
    b->pulse_count[sim] = count;
    b->pulse_period[sim] = period_steps;
    return IT_OK;
}

int it_batch_retime(it_batch *b) {
    if (!b) return bfail(IT_EINVAL, "batch is NULL");
    if (b->bstep != 0) return bfail(IT_ESTATE, "the time steps can only change before the first step");
    for (int s = 0; s < b->nsim; ++s) b->active[s] = 1;
    int rc = build_table(b);
    if (rc) return rc;
    const int ne = (int)b->tab.size();
    float *d_mx = nullptr;
    IT_CK(cudaMalloc(&d_mx, sizeof(float) * ne));
    batch_max_kernel<<<ne, 256, 0, b->stream>>>(b->d_sims, b->d_tab, b->state[0][0], b->state[0][1], d_mx);
    cudaError_t e = cudaGetLastError();
    std::vector<float> mx(ne);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx.data(), d_mx, sizeof(float) * ne, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d_mx);
    if (e != cudaSuccess) return cuda_fail(e, "batch peak density");
    int a = -1;
    for (int s = 0; s < b->nsim; ++s) {
        ++a;   // every simulation is active here: a indexes mfirst/mcount
        if (b->desc[s].dt_s > 0) continue;
        double npk = 0.0;
        for (int q = b->mfirst[a]; q < b->mfirst[a] + b->mcount[a]; ++q) npk = std::max(npk, (double)mx[q]);
        npk *= std::max(1, b->pulse_count[s]);   // a train can pile its pulses up
        if (!std::isfinite(npk)) return bfail(IT_EUNSTABLE, "simulation " + std::to_string(s) + " is not finite");
        const it_sim_desc &d = b->desc[s];
        it_params p = b->p;
        p.gap_cm = d.nz * d.dx_cm;
        p.voltage_V = d.voltage_V;
        p.n_peak_cm3 = npk;
        double dt = 0.0;
        rc = it_auto_dt(&p, d.dx_cm, &dt);
        if (rc) return rc;
        b->dt[s] = dt;
        coef_f32(&p, d.dx_cm, dt, &b->hs[s].cf);
    }
    IT_CK(cudaMemcpyAsync(b->d_sims, b->hs.data(), sizeof(BatchSim) * b->nsim, cudaMemcpyHostToDevice, b->stream));
    IT_CK(cudaStreamSynchronize(b->stream));
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return IT_OK;
}

int it_batch_set_chunk(it_batch *b, int64_t cells_per_block) {
    if (!b || cells_per_block < 256) return bfail(IT_EINVAL, "chunk must be at least 256 cells");
    b->chunk = cells_per_block;
    b->tab_dirty = true;
    return IT_OK;
}

int it_batch_autotune(it_batch *b, int32_t trial_steps, double *best_us) {
    if (!b) return bfail(IT_EINVAL, "batch is NULL");
    if (trial_steps < 2) return bfail(IT_EINVAL, "trial_steps must be at least 2");
    if (b->bstep != 0) return bfail(IT_ESTATE, "the launch shape is tuned before the first step");
    const int K = trial_steps + (trial_steps & 1);   // even: the state returns to set 0
    const size_t bytes = sizeof(float) * b->total;
    void *backup = nullptr;
    IT_CK(cudaMalloc(&backup, 2 * bytes));
    char *bk = (char *)backup;
    int rc = IT_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemcpyAsync(bk, b->state[0][0], bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(bk + bytes, b->state[0][1], bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "batch autotune set-up");
    const long long chunk0 = b->chunk;
    // TMA choice: 2 = the TMA kernel with two float4 per thread, 1 = with
    // one, 0 = the register kernel
    const int cps0 = b->vec_cps, tma0 = b->use_tma ? b->tma_ipt : 0;
    long long best_chunk = chunk0;
    int best_cps = cps0, best_tma = tma0;
    double best = 1e300;
    // the entry size only shapes the scalar kernel's entries: with no
    // simulation on that kernel a single size is timed
    bool any_scalar = false;
    for (int s = 0; s < b->nsim; ++s)
        if (b->active[s] && !(b->hs[s].nx % 4 == 0 && b->hs[s].nx <= 1024)) any_scalar = true;
    const std::vector<long long> chunks = any_scalar ? std::vector<long long>{4096LL, 16384LL, 65536LL}
                                                     : std::vector<long long>{chunk0};
    for (int tma : {2, 1, 0})
    for (int cps : {1, 2, 4, 8, 16, 32}) {
        for (long long chunk : chunks) {
            if (rc) break;
            b->use_tma = tma > 0;
            b->tma_ipt = tma == 2 ? 2 : 1;
            b->vec_cps = cps;
            b->chunk = chunk;
            rc = build_table(b);
            for (int q = 0; q < 2 && !rc; ++q) rc = launch_batched_step(b, q & 1);
            if (!rc && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "event");
            for (int q = 0; q < K && !rc; ++q) rc = launch_batched_step(b, q & 1);
            if (!rc && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "event");
            float ms = 0.f;
            if (!rc) {
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) rc = cuda_fail(e, "batch autotune timing");
            }
            // the trial steps changed the state: put the deposited state back
            if (cudaMemcpyAsync(b->state[0][0], bk, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
                cudaMemcpyAsync(b->state[0][1], bk + bytes, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
                rc = rc ? rc : cuda_fail(cudaGetLastError(), "batch autotune restore");
            if (!rc && ms * 1e3 / K < best) {
                best = ms * 1e3 / K;
                best_chunk = chunk;
                best_cps = cps;
                best_tma = tma;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    cudaFree(backup);
    // the chosen shape; the next table build also clears the trial tallies
    b->chunk = rc ? chunk0 : best_chunk;
    b->vec_cps = rc ? cps0 : best_cps;
    const int tma_sel = rc ? tma0 : best_tma;
    b->use_tma = tma_sel > 0;
    b->tma_ipt = tma_sel == 2 ? 2 : 1;
    b->tab_dirty = true;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (rc) return rc;
    if (best_us) *best_us = best;
    return IT_OK;
}

int it_batch_run(it_batch *b, double tol, int64_t max_steps, int64_t check_every, int64_t *launches) {
    if (!b) return bfail(IT_EINVAL, "batch is NULL");
    if (!(tol >= 0) || max_steps < 0 || check_every < 2) return bfail(IT_EINVAL, "bad argument");
    const int K = (int)(check_every + (check_every & 1));
    for (int s = 0; s < b->nsim; ++s)
        if (b->pulse_count[s] > 1 && b->pulse_period[s] % K != 0)
            return bfail(IT_EINVAL, "simulation " + std::to_string(s) + ": pulse period must be a multiple of the even check interval");
    std::vector<double> rel(8 * (size_t)b->nsim);
    IT_CK(cudaMemcpyAsync(rel.data(), b->d_rel, sizeof(double) * 8 * b->nsim, cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaStreamSynchronize(b->stream));
    int64_t nl = 0;
    std::vector<double> ind;
    for (;;) {
        if (b->tab_dirty) {
            int rc = build_table(b);
            if (rc) return rc;
        }
        // next pulse of a train: deposited at the start of its step
        bool deposited = false;
        for (size_t a = 0; a < b->sim_of.size(); ++a) {
            const int s = b->sim_of[a];
            const int done = b->pulse_done[s];
            if (done >= 1 && done < b->pulse_count[s] && b->steps[s] == (int64_t)done * b->pulse_period[s]) {
                const auto &pt = b->pulse_tracks[s];
                int rc = deposit_sim(b, s, pt.data(), (int64_t)(pt.size() / 4));
                if (rc) return rc;
                b->pulse_done[s] = done + 1;
                deposited = true;
            }
        }
        if (deposited) {
            IT_CK(cudaMemcpyAsync(rel.data(), b->d_rel, sizeof(double) * 8 * b->nsim, cudaMemcpyDeviceToHost, b->stream));
            IT_CK(cudaStreamSynchronize(b->stream));
        }
        // completion of every active simulation
        int rc = in_domain(b, ind);
        if (rc) return rc;
        bool changed = false;
        for (size_t a = 0; a < b->sim_of.size(); ++a) {
            const int s = b->sim_of[a];
            const double r = rel[8 * s] + rel[8 * s + 1];
            const double in = ind[2 * s] + ind[2 * s + 1];
            if (!std::isfinite(in)) return bfail(IT_EUNSTABLE, "simulation " + std::to_string(s) + " is not finite");
            const bool pending = b->pulse_done[s] >= 1 && b->pulse_done[s] < b->pulse_count[s];
            if (r <= 0 || (!pending && in / r < tol) || b->steps[s] >= max_steps) {
                b->active[s] = 0;
                changed = true;
            }
        }
        if (changed) {
            rc = build_table(b);
            if (rc) return rc;
        }
        if (b->tab.empty()) break;
        if (b->p.dt_ladder) {
            rc = ladder_batch(b);
            if (rc) return rc;
        }
        rc = run_segment(b, K);
        if (rc) return rc;
        nl += K;
        rc = fold(b);
        if (rc) return rc;
    }
    if (launches) *launches = nl;
    IT_CK(cudaStreamSynchronize(b->stream));
    return IT_OK;
}

int it_batch_tallies(it_batch *b, int32_t sim, it_tallies_t *t) {
    if (!b || !t || sim < 0 || sim >= b->nsim) return bfail(IT_EINVAL, "bad argument");
    double acc[NT], rel[8];
    IT_CK(cudaMemcpyAsync(acc, b->d_acc + (size_t)NT * sim, sizeof(acc), cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaMemcpyAsync(rel, b->d_rel + (size_t)8 * sim, sizeof(rel), cudaMemcpyDeviceToHost, b->stream));
    // in-domain charge and extreme densities of this simulation's current set
    const size_t cells = (size_t)b->hs[sim].nx * b->hs[sim].ny * b->hs[sim].nz;
    const int parity = (int)(b->steps[sim] & 1);
    constexpr int kMonBlocks = 64;
    double *d_mon = nullptr;
    IT_CK(cudaMalloc(&d_mon, sizeof(double) * NM * kMonBlocks));
    const double vol = b->dx[sim] * b->dx[sim] * b->dx[sim];
    int rc = launch_monitor_raw_f32(b->state[parity][0] + b->hs[sim].off, b->state[parity][1] + b->hs[sim].off,
                                    cells, vol, d_mon, kMonBlocks, b->stream);
    double mon[NM * kMonBlocks];
    if (rc == IT_OK) {
        cudaError_t e = cudaMemcpyAsync(mon, d_mon, sizeof(mon), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch tallies");
    }
    cudaFree(d_mon);
    if (rc) return rc;
    std::memset(t, 0, sizeof(*t));
    for (int s = 0; s < 2; ++s) {
        double sum = 0, mn = INFINITY, mx = -INFINITY;
        for (int q = 0; q < kMonBlocks; ++q) {
            sum += mon[q * NM + s];
            mn = std::min(mn, mon[q * NM + 2 + s]);
            mx = std::max(mx, mon[q * NM + 4 + s]);
        }
        t->in_domain[s] = sum;
        t->n_min[s] = mn;
        t->n_max[s] = mx;
    }
    t->recombined = acc[0];
    t->collected_anode[0] = acc[1]; t->collected_anode[1] = acc[2];
    t->collected_cathode[0] = acc[3]; t->collected_cathode[1] = acc[4];
    t->lost_lateral[0] = acc[5]; t->lost_lateral[1] = acc[6];
    t->space_charge[0] = acc[7]; t->space_charge[1] = acc[8];
    t->released[0] = rel[0]; t->released[1] = rel[1];
    const double r = rel[0] + rel[1];
    t->f = r > 0 ? (acc[1] + acc[2] + acc[3] + acc[4]) / r : NAN;
    t->steps = b->steps[sim];
    t->dt_s = b->dt[sim];
    t->t_s = b->t_s[sim];
    return IT_OK;
}

int it_batch_get_density(it_batch *b, int32_t sim, int species, void *dst, size_t bytes) {
    if (!b || !dst || sim < 0 || sim >= b->nsim || (species != 0 && species != 1)) return bfail(IT_EINVAL, "bad argument");
    const size_t cells = (size_t)b->hs[sim].nx * b->hs[sim].ny * b->hs[sim].nz;
    if (bytes != cells * sizeof(float)) return bfail(IT_EINVAL, "bytes must equal cells * 4");
    const int parity = (int)(b->steps[sim] & 1);
    IT_CK(cudaMemcpyAsync(dst, b->state[parity][species] + b->hs[sim].off, bytes, cudaMemcpyDeviceToHost, b->stream));
    IT_CK(cudaStreamSynchronize(b->stream));
    return IT_OK;
}

int it_batch_destroy(it_batch *b) {
    batch_free(b);
    return IT_OK;
}

}  // extern "C"
