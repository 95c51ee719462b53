// it_kernels.cu -- deposition, the simple step kernel, monitor and tally
// reduction kernels.
//
// Deposition follows Eqs. (linear_density), (Gaussian), (created): a track
// parallel to E with N0 = LET/W ions per cm and radial profile
// N0/(pi b^2) exp(-r^2/b^2), integrated over each cell, identical on every z
// plane.  The step is the Appendix scheme (Lax-Wendroff drift along z, FTCS
// diffusion on three axes, -alpha n+ n- from the old level), written in flux
// form so the tallies of what crosses the electrode faces close the charge
// balance.
#include <cmath>

#include "it_device.cuh"
#include "it_internal.cuh"

namespace itk {

// ---------------------------------------------------------------------------
// simple step: one thread per cell, neighbours read through L1/L2
// ---------------------------------------------------------------------------
template <typename T, bool PERIODIC>
__global__ void __launch_bounds__(256)
step_simple_kernel(const T *__restrict__ ip, const T *__restrict__ im, T *__restrict__ op,
                   T *__restrict__ om, int nx, int ny, int nz, Coef<T> c,
                   double *__restrict__ slots) {
    __shared__ double red[32 * 9];
    const size_t plane = (size_t)nx * ny;
    const size_t total = plane * nz;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx);
        const size_t r = idx / nx;
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const size_t ixm = (i > 0) ? idx - 1 : idx + (nx - 1);
        const size_t ixp = (i < nx - 1) ? idx + 1 : idx - (nx - 1);
        const size_t iym = (j > 0) ? idx - nx : idx + (size_t)(ny - 1) * nx;
        const size_t iyp = (j < ny - 1) ? idx + nx : idx - (size_t)(ny - 1) * nx;
        const T p0 = ip[idx], m0 = im[idx];
        const T rr = p0 * m0;
        acc[0] += (double)rr;
        const int cx = (i == 0) + (i == nx - 1);
        const int cy = (j == 0) + (j == ny - 1);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T *in = s ? im : ip;
            const T n0 = s ? m0 : p0;
            const T xm = (PERIODIC || i > 0) ? in[ixm] : T(0);
            const T xp = (PERIODIC || i < nx - 1) ? in[ixp] : T(0);
            const T ym = (PERIODIC || j > 0) ? in[iym] : T(0);
            const T yp = (PERIODIC || j < ny - 1) ? in[iyp] : T(0);
            const T zm = (k > 0) ? in[idx - plane] : T(0);
            const T zp = (k < nz - 1) ? in[idx + plane] : T(0);
            T v = upd7(n0, xm, xp, ym, yp, zm, zp, rr, c.wx[s], c.wzm[s], c.wzp[s], c.adt);
            if (c.sc_on) {
                v = add_sc(v, c.sc[s], n0, p0, m0);
                acc[7 + s] += (double)(n0 * (p0 - m0));
            }
            (s ? om : op)[idx] = v;
            if (k == 0) acc[1 + s] += (double)n0;
            if (k == nz - 1) acc[3 + s] += (double)n0;
            if (!PERIODIC && (cx | cy))
                acc[5 + s] += (double)n0 * (cx * c.latx_f[s] + cy * c.laty_f[s]);
        }
    }
    block_sum<9>(acc, red);
    if (threadIdx.x == 0) {
        double *sl = slots + (size_t)blockIdx.x * NT;
        sl[0] += acc[0] * c.rec_f;
        sl[1] += acc[1] * c.anode_f[0];
        sl[2] += acc[2] * c.anode_f[1];
        sl[3] += acc[3] * c.cathode_f[0];
        sl[4] += acc[4] * c.cathode_f[1];
        sl[5] += acc[5];
        sl[6] += acc[6];
        sl[7] += acc[7] * c.sc_f[0];
        sl[8] += acc[8] * c.sc_f[1];
    }
}

int simple_grid(const it_ctx *c) {
    const size_t blocks = (c->g.cells() + 255) / 256;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t cap = (size_t)sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int launch_step_simple(it_ctx *c, cudaStream_t s) {
    const int nb = c->nslots;
    const int cur = c->cur, nxt = cur ^ 1;
    if (c->prec == IT_FP32) {
        auto *ip = (const float *)c->n[cur][0], *im = (const float *)c->n[cur][1];
        auto *op = (float *)c->n[nxt][0], *om = (float *)c->n[nxt][1];
        if (c->p.lateral_bc == IT_PERIODIC)
            step_simple_kernel<float, true><<<nb, 256, 0, s>>>(ip, im, op, om, c->g.nx, c->g.ny, c->g.nz, c->cf, c->d_slots);
        else
            step_simple_kernel<float, false><<<nb, 256, 0, s>>>(ip, im, op, om, c->g.nx, c->g.ny, c->g.nz, c->cf, c->d_slots);
    } else {
        auto *ip = (const double *)c->n[cur][0], *im = (const double *)c->n[cur][1];
        auto *op = (double *)c->n[nxt][0], *om = (double *)c->n[nxt][1];
        if (c->p.lateral_bc == IT_PERIODIC)
            step_simple_kernel<double, true><<<nb, 256, 0, s>>>(ip, im, op, om, c->g.nx, c->g.ny, c->g.nz, c->cd, c->d_slots);
        else
            step_simple_kernel<double, false><<<nb, 256, 0, s>>>(ip, im, op, om, c->g.nx, c->g.ny, c->g.nz, c->cd, c->d_slots);
    }
    IT_CK(cudaGetLastError());
    c->cur = nxt;
    return IT_OK;
}

// The simple step on caller-given FP32 arrays with a caller-given slot array
// of nblocks x NT doubles (one block per slot, grid-stride over the cells).
int launch_step_simple_raw_f32(const float *ip, const float *im, float *op, float *om, int nx, int ny, int nz,
                               const Coef<float> &cf, bool periodic, double *slots, int nblocks, cudaStream_t s) {
    if (periodic)
        step_simple_kernel<float, true><<<nblocks, 256, 0, s>>>(ip, im, op, om, nx, ny, nz, cf, slots);
    else
        step_simple_kernel<float, false><<<nblocks, 256, 0, s>>>(ip, im, op, om, nx, ny, nz, cf, slots);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// ---------------------------------------------------------------------------
// monitor: in-domain ions and extreme densities of the current state
// ---------------------------------------------------------------------------
// Per-thread accumulation of one cell of each species into T partial sums
// and extremes; the partials are moved to FP64 by flush(), which callers run
// once per at most 32 cells outside the per-cell code (FP64 is slow on this
// GPU: an FP64 add in the per-cell path, even a predicated one, would bound
// the kernel).
template <typename T>
struct MonAcc {
    double sum[2] = {0.0, 0.0};
    T part[2] = {0, 0};
    T mn[2] = {(T)INFINITY, (T)INFINITY}, mx[2] = {(T)-INFINITY, (T)-INFINITY};
    __device__ __forceinline__ void add(T a, T b) {
        part[0] += a; part[1] += b;          // a NaN propagates into the sums
        mn[0] = a < mn[0] ? a : mn[0]; mn[1] = b < mn[1] ? b : mn[1];
        mx[0] = a > mx[0] ? a : mx[0]; mx[1] = b > mx[1] ? b : mx[1];
    }
    __device__ __forceinline__ void flush() {
        sum[0] += (double)part[0]; sum[1] += (double)part[1];
        part[0] = part[1] = 0;
    }
};

// In-domain sums and extremes of both species, one row of NM values per CTA.
// FP32 states on 16-byte boundaries are read as float4, four loads of each
// species in flight per thread, and summed in FP32 over 32 cells (two
// rounds of four float4) before FP64; other cells are read one by one and
// summed in T over up to 32 cells.
template <typename T>
__global__ void __launch_bounds__(256)
monitor_kernel(const T *__restrict__ ip, const T *__restrict__ im, size_t total, double vol,
               double *__restrict__ mon) {
    __shared__ double red[32 * 2];
    __shared__ double rmin[32 * 2], rmax[32 * 2];
    MonAcc<T> acc;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    const bool vec = sizeof(T) == 4 && (((uintptr_t)ip | (uintptr_t)im) & 15) == 0;
    if (vec) {
        const size_t n4 = total / 4;
        const float4 *p4 = reinterpret_cast<const float4 *>(ip);
        const float4 *m4 = reinterpret_cast<const float4 *>(im);
        size_t q = tid;
        bool more = true;
        while (more) {
            // one round: up to two groups of four float4 per species (32 cells)
            for (int g = 0; g < 2; ++g) {
                if (q + 3 * nthr >= n4) { more = false; break; }
                float4 a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = __ldcs(p4 + q + u * nthr);
                    b[u] = __ldcs(m4 + q + u * nthr);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc.add(a[u].x, b[u].x); acc.add(a[u].y, b[u].y);
                    acc.add(a[u].z, b[u].z); acc.add(a[u].w, b[u].w);
                }
                q += 4 * nthr;
            }
            acc.flush();
        }
        for (; q < n4; q += nthr) {   // fewer than four float4 left per thread
            const float4 a = __ldcs(p4 + q), b = __ldcs(m4 + q);
            acc.add(a.x, b.x); acc.add(a.y, b.y); acc.add(a.z, b.z); acc.add(a.w, b.w);
        }
        acc.flush();
        done = n4 * 4;
    }
    {
        int n = 0;
        for (size_t idx = done + tid; idx < total; idx += nthr) {
            acc.add(ip[idx], im[idx]);
            if (++n == 32) { acc.flush(); n = 0; }
        }
        acc.flush();
    }
    double sum[2] = {acc.sum[0], acc.sum[1]};
    double mn[2] = {(double)acc.mn[0], (double)acc.mn[1]}, mx[2] = {(double)acc.mx[0], (double)acc.mx[1]};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[q] = fmin(mn[q], __shfl_down_sync(0xffffffffu, mn[q], o));
            mx[q] = fmax(mx[q], __shfl_down_sync(0xffffffffu, mx[q], o));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        rmin[warp * 2] = mn[0]; rmin[warp * 2 + 1] = mn[1];
        rmax[warp * 2] = mx[0]; rmax[warp * 2 + 1] = mx[1];
    }
    block_sum<2>(sum, red);   // contains the __syncthreads for rmin/rmax too
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int w = 1; w < nw; ++w) {
            mn[0] = fmin(mn[0], rmin[w * 2]); mn[1] = fmin(mn[1], rmin[w * 2 + 1]);
            mx[0] = fmax(mx[0], rmax[w * 2]); mx[1] = fmax(mx[1], rmax[w * 2 + 1]);
        }
        double *m = mon + (size_t)blockIdx.x * NM;
        m[0] = sum[0] * vol; m[1] = sum[1] * vol;
        m[2] = mn[0]; m[3] = mn[1]; m[4] = mx[0]; m[5] = mx[1];
    }
}

int launch_monitor(it_ctx *c, cudaStream_t s) {
    const double vol = c->dx * c->dx * c->dx;
    const int cur = c->cur;
    if (c->prec == IT_FP32)
        monitor_kernel<float><<<c->nmon, 256, 0, s>>>((const float *)c->n[cur][0], (const float *)c->n[cur][1],
                                                     c->g.cells(), vol, c->d_mon);
    else
        monitor_kernel<double><<<c->nmon, 256, 0, s>>>((const double *)c->n[cur][0], (const double *)c->n[cur][1],
                                                      c->g.cells(), vol, c->d_mon);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// monitor over caller-given FP32 arrays into nblocks x NM values
int launch_monitor_raw_f32(const float *p, const float *m, size_t cells, double vol, double *mon, int nblocks,
                           cudaStream_t s) {
    monitor_kernel<float><<<nblocks, 256, 0, s>>>(p, m, cells, vol, mon);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// ---------------------------------------------------------------------------
// finalize: fixed-order sums of the per-CTA slots and monitor values
//   out[0..NT) tallies, out[NT..NT+NM) monitor, out[NT+NM..+2) released
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
finalize_kernel(const double *__restrict__ slots, int nslots, const double *__restrict__ mon,
                int nmon, const double *__restrict__ acc, const int *__restrict__ err, double *__restrict__ out) {
    __shared__ double red[32 * (NT + 2)];
    __shared__ double rmin[32 * 2], rmax[32 * 2];
    double v[NT + 2];
#pragma unroll
    for (int q = 0; q < NT + 2; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nslots; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NT; ++q) v[q] += slots[(size_t)b * NT + q];
    }
    double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nmon; b += blockDim.x) {
        v[NT] += mon[(size_t)b * NM + 0];
        v[NT + 1] += mon[(size_t)b * NM + 1];
        mn[0] = fmin(mn[0], mon[(size_t)b * NM + 2]); mn[1] = fmin(mn[1], mon[(size_t)b * NM + 3]);
        mx[0] = fmax(mx[0], mon[(size_t)b * NM + 4]); mx[1] = fmax(mx[1], mon[(size_t)b * NM + 5]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[q] = fmin(mn[q], __shfl_down_sync(0xffffffffu, mn[q], o));
            mx[q] = fmax(mx[q], __shfl_down_sync(0xffffffffu, mx[q], o));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        rmin[warp * 2] = mn[0]; rmin[warp * 2 + 1] = mn[1];
        rmax[warp * 2] = mx[0]; rmax[warp * 2 + 1] = mx[1];
    }
    block_sum<NT + 2>(v, red);
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int w = 1; w < nw; ++w) {
            mn[0] = fmin(mn[0], rmin[w * 2]); mn[1] = fmin(mn[1], rmin[w * 2 + 1]);
            mx[0] = fmax(mx[0], rmax[w * 2]); mx[1] = fmax(mx[1], rmax[w * 2 + 1]);
        }
        for (int q = 0; q < NT; ++q) out[q] = v[q];
        out[NT + 0] = v[NT]; out[NT + 1] = v[NT + 1];
        out[NT + 2] = mn[0]; out[NT + 3] = mn[1]; out[NT + 4] = mx[0]; out[NT + 5] = mx[1];
        out[NT + NM + 0] = acc[0];
        out[NT + NM + 1] = acc[1];
        out[NT + NM + 2] = (double)*err;
    }
}

int launch_finalize(it_ctx *c, cudaStream_t s) {
    finalize_kernel<<<1, 256, 0, s>>>(c->d_slots, c->nslots, c->d_mon, c->nmon, c->d_acc, c->d_err, c->d_out);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// ---------------------------------------------------------------------------
// deposition
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long floor_div(long long a, long long n) {
    return (a >= 0) ? a / n : -((-a + n - 1) / n);
}

// Per track and axis: the fraction of the 1D Gaussian factor
// exp(-u^2/b^2)/(sqrt(pi) b) that falls in each cell, summed over the
// periodic images of the cell inside the window +-ceil(6 b/dx) around the
// centre cell (absorbing faces: only the cell itself, if inside).
__global__ void deposit_tables_kernel(const double *__restrict__ tr, double dx, int nx, int ny,
                                      int periodic, double *__restrict__ wx, double *__restrict__ wy) {
    const long long t = blockIdx.x;
    const int axis = blockIdx.y;
    const int n = axis ? ny : nx;
    const double ctr = tr[t * 4 + axis];
    const double b = tr[t * 4 + 3];
    const long long w = (long long)ceil(6.0 * b / dx);
    const long long ic = (long long)floor(ctr / dx);
    const long long lo = ic - w, hi = ic + w;
    double *out = axis ? (wy + t * ny) : (wx + t * nx);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double sum = 0.0;
        if (periodic) {
            long long ii = i + n * (-floor_div(-(lo - i), n));   // first image >= lo
            for (; ii <= hi; ii += n)
                sum += 0.5 * (erf(((double)(ii + 1) * dx - ctr) / b) - erf(((double)ii * dx - ctr) / b));
        } else if (i >= lo && i <= hi) {
            sum = 0.5 * (erf(((double)(i + 1) * dx - ctr) / b) - erf(((double)i * dx - ctr) / b));
        }
        out[i] = sum;
    }
}

// Does the deposit window of a track (+-w cells around cell ic, wrapped on a
// periodic axis of n cells) reach the cells [t0, t0 + tn)?  Conservative: a
// track that only touches zero weights is harmless (it adds exact zeros).
__device__ __forceinline__ bool window_hits(long long ic, long long w, int t0, int tn, int n, bool periodic) {
    if (periodic) {
        if (2 * w + 1 >= n) return true;
        long long d = ((long long)t0 - (ic - w)) % n;
        if (d < 0) d += n;
        return d <= 2 * w || d + tn - 1 >= n;
    }
    return ic + w >= t0 && ic - w <= t0 + tn - 1;
}

constexpr int DEP_TILE = 16;      // 16 x 16 cells per CTA
constexpr int DEP_LIST = 1024;    // tracks gathered per pass

// plane[j][i] = sum_t N0_t wx[t][i] wy[t][j] / dx^2, tracks in index order.
// Each CTA first lists (in index order) the tracks whose window reaches its
// tile, then every cell sums over that list; tracks that miss the tile only
// contribute zeros, so the per-cell sum is the same as over all tracks.
// part[blockIdx] receives the tile's sum of the plane (FP64).
__global__ void __launch_bounds__(DEP_TILE *DEP_TILE)
deposit_plane_kernel(const double *__restrict__ tr, const double *__restrict__ wx, const double *__restrict__ wy,
                     long long nt, int nx, int ny, double dx, int periodic, double inv_dx2, double inv_W,
                     double *__restrict__ plane, double *__restrict__ part) {
    __shared__ int list[DEP_LIST];
    __shared__ int wcount[DEP_TILE * DEP_TILE / 32];
    __shared__ int nlist;
    __shared__ double red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = blockIdx.x * DEP_TILE, j0 = blockIdx.y * DEP_TILE;
    const int tnx = min(DEP_TILE, nx - i0), tny = min(DEP_TILE, ny - j0);
    const int i = i0 + (tid % DEP_TILE), j = j0 + (tid / DEP_TILE);
    const bool inside = (tid % DEP_TILE) < tnx && (tid / DEP_TILE) < tny;
    double sum = 0.0;
    for (long long base = 0; base < nt;) {
        if (tid == 0) nlist = 0;
        __syncthreads();
        // gather up to DEP_LIST candidates in index order, 256 tracks per round
        long long t0 = base;
        for (; t0 < nt; t0 += blockDim.x) {
            const long long t = t0 + tid;
            bool hit = false;
            if (t < nt) {
                const double b = tr[t * 4 + 3];
                const long long w = (long long)ceil(6.0 * b / dx);
                hit = window_hits((long long)floor(tr[t * 4] / dx), w, i0, tnx, nx, periodic != 0) &&
                      window_hits((long long)floor(tr[t * 4 + 1] / dx), w, j0, tny, ny, periodic != 0);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) wcount[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                if (q < warp) before += wcount[q];
                total += wcount[q];
            }
            const int start = nlist;
            if (total > DEP_LIST - start) {   // list full: stop before this round, take it next pass
                __syncthreads();
                break;
            }
            if (hit) list[start + before + __popc(bal & ((1u << lane) - 1u))] = (int)t;
            __syncthreads();
            if (tid == 0) nlist = start + total;
            __syncthreads();
        }
        const int n = nlist;
        if (inside) {
            for (int q = 0; q < n; ++q) {
                const long long t = list[q];
                const double a = wx[t * nx + i];
                if (a == 0.0) continue;
                const double bb = wy[t * ny + j];
                if (bb == 0.0) continue;
                const double N0 = tr[t * 4 + 2] * 1e7 * inv_W;   // ions per cm
                sum += N0 * a * bb;
            }
        }
        base = t0;
        __syncthreads();
    }
    const double v = sum * inv_dx2;
    if (inside) plane[(size_t)j * nx + i] = v;
    double r[1] = {inside ? v : 0.0};
    block_sum<1>(r, red);
    if (tid == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = r[0];
}

// n += plane on every z plane.  Thread = V adjacent columns (float4 when the
// state is FP32 and nx % 4 == 0) over a chunk of DEP_KCHUNK planes
// (blockIdx.y); columns the deposit did not reach are skipped.  FP32 states
// add the plane value rounded to FP32 (n + float(plane), one FP32 addition:
// FP64 arithmetic is slow on this GPU and the two roundings stay within an
// ulp of the exact sum); FP64 states add it exactly in FP64.
constexpr int DEP_KCHUNK = 8;
template <typename T, int V>
__global__ void __launch_bounds__(256)
deposit_apply_kernel(T *__restrict__ p, T *__restrict__ m, const double *__restrict__ plane, size_t plane_n,
                     int nz) {
    const size_t c0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (c0 >= plane_n) return;
    double a[V];
    bool any = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        a[v] = plane[c0 + v];
        any |= a[v] != 0.0;
    }
    if (!any) return;   // x + 0 == x: nothing to write
    const int k0 = blockIdx.y * DEP_KCHUNK, k1 = min(nz, k0 + DEP_KCHUNK);
    if constexpr (V == 4) {
        const float4 af = make_float4(__double2float_rn(a[0]), __double2float_rn(a[1]), __double2float_rn(a[2]),
                                      __double2float_rn(a[3]));
        float4 *p4 = reinterpret_cast<float4 *>(p), *m4 = reinterpret_cast<float4 *>(m);
        for (int k = k0; k < k1; ++k) {
            const size_t i4 = ((size_t)k * plane_n + c0) / 4;
            float4 x = p4[i4], y = m4[i4];
            x.x = __fadd_rn(x.x, af.x); x.y = __fadd_rn(x.y, af.y); x.z = __fadd_rn(x.z, af.z); x.w = __fadd_rn(x.w, af.w);
            y.x = __fadd_rn(y.x, af.x); y.y = __fadd_rn(y.y, af.y); y.z = __fadd_rn(y.z, af.z); y.w = __fadd_rn(y.w, af.w);
            p4[i4] = x;
            m4[i4] = y;
        }
    } else if constexpr (sizeof(T) == 4) {
        const float af = __double2float_rn(a[0]);
        for (int k = k0; k < k1; ++k) {
            const size_t idx = (size_t)k * plane_n + c0;
            p[idx] = __fadd_rn(p[idx], af);
            m[idx] = __fadd_rn(m[idx], af);
        }
    } else {
        for (int k = k0; k < k1; ++k) {
            const size_t idx = (size_t)k * plane_n + c0;
            p[idx] += a[0];
            m[idx] += a[0];
        }
    }
}

// released += sum(tile sums) * dx^2 * (nz dx) for both species, fixed order
__global__ void __launch_bounds__(256)
deposit_released_kernel(const double *__restrict__ part, size_t n, double factor, double *__restrict__ acc) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) v[0] += part[q];
    block_sum<1>(v, red);
    if (threadIdx.x == 0) {
        acc[0] += v[0] * factor;
        acc[1] += v[0] * factor;
    }
}

int launch_deposit(it_ctx *c, int64_t n, cudaStream_t s) {
    if (n <= 0) return IT_OK;
    const int nx = c->g.nx, ny = c->g.ny;
    const bool periodic = c->p.lateral_bc == IT_PERIODIC;
    dim3 gt((unsigned)n, 2);
    deposit_tables_kernel<<<gt, 128, 0, s>>>(c->d_tracks, c->dx, nx, ny, periodic, c->d_wx, c->d_wy);
    IT_CK(cudaGetLastError());
    const long long pn = (long long)nx * ny;
    dim3 gp((nx + DEP_TILE - 1) / DEP_TILE, (ny + DEP_TILE - 1) / DEP_TILE);
    const size_t nparts = (size_t)gp.x * gp.y;
    // the tile sums go after the plane in the same scratch buffer
    double *part = c->d_plane + pn;
    deposit_plane_kernel<<<gp, DEP_TILE * DEP_TILE, 0, s>>>(c->d_tracks, c->d_wx, c->d_wy, n, nx, ny, c->dx,
                                                            periodic ? 1 : 0, 1.0 / (c->dx * c->dx),
                                                            1.0 / c->p.W_eV, c->d_plane, part);
    IT_CK(cudaGetLastError());
    const unsigned kchunks = (unsigned)((c->g.nz + DEP_KCHUNK - 1) / DEP_KCHUNK);
    if (c->prec == IT_FP32 && nx % 4 == 0)
        deposit_apply_kernel<float, 4><<<dim3((unsigned)((pn / 4 + 255) / 256), kchunks), 256, 0, s>>>(
            (float *)c->n[c->cur][0], (float *)c->n[c->cur][1], c->d_plane, (size_t)pn, c->g.nz);
    else if (c->prec == IT_FP32)
        deposit_apply_kernel<float, 1><<<dim3((unsigned)((pn + 255) / 256), kchunks), 256, 0, s>>>(
            (float *)c->n[c->cur][0], (float *)c->n[c->cur][1], c->d_plane, (size_t)pn, c->g.nz);
    else
        deposit_apply_kernel<double, 1><<<dim3((unsigned)((pn + 255) / 256), kchunks), 256, 0, s>>>(
            (double *)c->n[c->cur][0], (double *)c->n[c->cur][1], c->d_plane, (size_t)pn, c->g.nz);
    IT_CK(cudaGetLastError());
    const double factor = c->dx * c->dx * (c->dx * c->g.nz);
    deposit_released_kernel<<<1, 256, 0, s>>>(part, nparts, factor, c->d_acc);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// ---------------------------------------------------------------------------
// tracks at an angle theta to the field (Fig. setup (a))
// ---------------------------------------------------------------------------

// Sum of the cell weights (erf(hi/w) - erf(lo/w))/2 of a profile of width w
// centred at c over the images of cell q in the window [lo_c, hi_c] (cell
// indices, unwrapped): every q + m n inside it when periodic, q itself when not.
__device__ __forceinline__ double image_weights(int q, int n, int lo_c, int hi_c, double c, double w, double dx,
                                                bool periodic) {
    int m0 = 0, m1 = 0;
    if (periodic) {
        // smallest m with q + m n >= lo_c (a ceiling) and largest with
        // q + m n <= hi_c (a floor); C division truncates toward zero
        const int a = lo_c - q, bb = hi_c - q;
        m0 = a >= 0 ? (a + n - 1) / n : -((-a) / n);
        m1 = bb >= 0 ? bb / n : -((-bb + n - 1) / n);
    } else if (q < lo_c || q > hi_c) {
        return 0.0;
    }
    double s = 0.0;
    for (int m = m0; m <= m1; ++m) {
        const double lo = (double)(q + m * n) * dx;
        s += 0.5 * (erf((lo + dx - c) / w) - erf((lo - c) / w));
    }
    return s;
}

// One thread per cell (grid-stride, fixed grid), the tracks in order.  Track
// record [5]: x0, y0, N0 (ions/cm), b, theta.  In the plane of cell centres
// z_k the tilted column's cross-section is the Gaussian of width b/cos(theta)
// in x centred at x0 + (z_k - d/2) tan(theta) and of width b in y:
// (N0/cos) wx wy / dx^2 with the cell weights wx, wy over +-ceil(6 w/dx)
// cells (images summed when periodic).  Within cos(theta) dx / b < 1e-3 of
// parallel to the electrodes the track is one column through the box and wx
// is the cell-centre value dx exp(-u^2/b^2)/(sqrt(pi) b/cos) with
// u = (x - x0) cos - (z_k - d/2) sin: N0/(sqrt(pi) b) exp(-u^2/b^2) wy/dx.
// FP32 states add the FP64 sum rounded once, as the parallel deposit does.
// Each block writes its FP64 sum of the added densities (fixed order).
template <typename T>
__global__ void __launch_bounds__(256)
deposit_angled_kernel(const double *__restrict__ tr, int n, int nx, int ny, int nz, double dx, int periodic,
                      T *__restrict__ p, T *__restrict__ m, double *__restrict__ part) {
    __shared__ double red[32];
    const double zmid = 0.5 * nz * dx;
    const double sqrt_pi = 1.7724538509055160272981674833411;
    const size_t cells = (size_t)nx * ny * nz;
    double bsum[1] = {0.0};
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < cells;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % (size_t)nx);
        const int j = (int)((idx / (size_t)nx) % (size_t)ny);
        const int k = (int)(idx / ((size_t)nx * ny));
        const double zk = (k + 0.5) * dx;
        double v = 0.0;
        for (int t = 0; t < n; ++t) {
            const double x0 = tr[5 * t], y0 = tr[5 * t + 1], N0 = tr[5 * t + 2], b = tr[5 * t + 3];
            const double th = tr[5 * t + 4];
            const int wy = (int)ceil(6.0 * b / dx), jc = (int)floor(y0 / dx);
            const double sy = image_weights(j, ny, jc - wy, jc + wy, y0, b, dx, periodic);
            if (sy == 0.0) continue;
            const double c = cos(th), sn = sin(th);
            if (c * dx / b < 1e-3) {
                const double u = ((i + 0.5) * dx - x0) * c - (zk - zmid) * sn;
                v += N0 / (sqrt_pi * b) * exp(-(u * u) / (b * b)) * sy / dx;
            } else {
                const double xc = x0 + (zk - zmid) * sn / c;
                const int wx = (int)ceil(6.0 * b / (dx * c)), ic = (int)floor(xc / dx);
                const double sx = image_weights(i, nx, ic - wx, ic + wx, xc, b / c, dx, periodic);
                v += (N0 / c) * sx * sy / (dx * dx);
            }
        }
        if (v != 0.0) {
            if constexpr (sizeof(T) == 4) {
                const float vf = __double2float_rn(v);
                p[idx] = __fadd_rn(p[idx], vf);
                m[idx] = __fadd_rn(m[idx], vf);
            } else {
                p[idx] += v;
                m[idx] += v;
            }
            bsum[0] += v;
        }
    }
    block_sum<1>(bsum, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum[0];
}

int launch_deposit_angled(it_ctx *c, const double *d_tr, int64_t n, double *d_part, int nblocks, cudaStream_t s) {
    if (n <= 0) return IT_OK;
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    const int per = c->p.lateral_bc == IT_PERIODIC ? 1 : 0;
    if (c->prec == IT_FP32)
        deposit_angled_kernel<float><<<nblocks, 256, 0, s>>>(d_tr, (int)n, nx, ny, nz, c->dx, per,
                                                             (float *)c->n[c->cur][0], (float *)c->n[c->cur][1],
                                                             d_part);
    else
        deposit_angled_kernel<double><<<nblocks, 256, 0, s>>>(d_tr, (int)n, nx, ny, nz, c->dx, per,
                                                              (double *)c->n[c->cur][0],
                                                              (double *)c->n[c->cur][1], d_part);
    IT_CK(cudaGetLastError());
    const double vol = c->dx * c->dx * c->dx;
    deposit_released_kernel<<<1, 256, 0, s>>>(d_part, (size_t)nblocks, vol, c->d_acc);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

int launch_zero(void *p, size_t bytes, cudaStream_t s) {
    IT_CK(cudaMemsetAsync(p, 0, bytes, s));
    return IT_OK;
}

}  // namespace itk
