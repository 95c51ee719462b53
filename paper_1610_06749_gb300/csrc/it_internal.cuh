// it_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "iontracks.h"

namespace itk {

// Tally slots every step kernel writes per CTA (FP64, accumulated over all
// steps by the CTA that owns the slot, so the fixed-order final reduction is
// deterministic):
//   0 recombined ion pairs, 1/2 anode +/-, 3/4 cathode +/-, 5/6 lateral +/-,
//   7/8 ions added by the space-charge term +/- (9 unused)
constexpr int NT = 10;
// Monitor values of the current state per CTA: in-domain +/- (ions),
// min +/-, max +/- (densities).
constexpr int NM = 6;
// finalize output: NT tallies, NM monitor values, released +/-, error flag
constexpr int NOUT = NT + NM + 3;

// Update weights of one species, for the increment in flux form
//   n' = n + [wx ((x- + x+) + (y- + y+) - 4 n) + wzm (z- - n) + wzp (z+ - n)
//             - adt n+ n-]
// (wx = wy: the cells are cubes); wzm multiplies the difference to the
// neighbour at k-1, wzp the one at k+1.  The transport part sums to zero over
// the grid for any weights, so each weight is its nearest value in T and
// charge is conserved in real arithmetic (only per-operation rounding
// remains).
template <typename T>
struct Coef {
    T wx[2], wy[2], wzm[2], wzp[2];
    T adt;            // alpha * dt
    T sc[2];          // space charge: the update adds sc[s] n_s (n+ - n-);
                      // sc = -dt mu+ q/eps0 for n+, +dt mu- q/eps0 for n-
    int sc_on;        // 1: the space-charge term is on
    // FP64 factors that turn per-CTA sums into ions (weights as rounded to T)
    double rec_f;     // adt * vol
    double anode_f[2];    // wzp * vol  (cell k=0 sends wzp to the ghost k=-1)
    double cathode_f[2];  // wzm * vol  (cell k=nz-1 sends wzm to the ghost k=nz)
    double latx_f[2], laty_f[2];
    double sc_f[2];   // sc * vol (tally of the space-charge term)
};

struct Grid {
    int nx, ny, nz;
    size_t plane() const { return (size_t)nx * ny; }
    size_t cells() const { return plane() * nz; }
};

// Launch shape of the z-march kernel: tiles of TY full-width rows; each CTA
// takes a contiguous range of (tile, plane) pairs and streams the planes
// through an S-deep ring of shared-memory slots by TMA.
struct ZmConf {
    int TY;           // rows per tile (divides ny)
    int nzc;          // CTAs in the grid (each takes a contiguous range of tile-planes)
    int ntile;        // ny / TY
    int S;            // ring depth (>= 3)
    int bx;           // row width a block holds (nx; 256 for the 3-D maps of nx > 256)
    int nbx;          // nx / bx
    int xs;           // 1: 3-D maps; nx / 256 > 1: 4-D maps that split a row into xs
                      // 256-float pieces, so one box carries whole rows (bx = nx)
    int reg_top, reg_main, reg_bot;   // float offsets of the halo/main rows in a block
    int blk;          // floats per (species, x-box) block, 128-byte multiple
    int slot;         // floats per slot = 2 * nbx * blk
    unsigned tx_bytes;   // bytes TMA delivers per slot
    size_t smem;      // dynamic shared memory per CTA
    int threads;      // 256
    int ctas_per_sm;
    long long wait_cycles;   // SM cycles a ring wait may take before it is declared lost
    int withhold;            // test hook: 1 = the first ring load is never issued
};

// Launch shape of the two-steps-per-launch z-march kernel: tiles of TY
// full-width rows, one float4 item per thread of the tile (TY * nx/4 ==
// threads); a ring slot holds TY + 4 rows of both species (two halo rows
// above and below), the intermediate level lives in two shared-memory planes
// of TY + 2 rows.
struct Zm2Conf {
    int TY, ntile, S, bx, nbx;
    int reg_top, reg_main, reg_bot;   // float offsets of the 2-row halos and TY rows in a ring block
    int blk, slot;                    // floats per (species, x-box) ring block / per ring slot
    int mblk, mslot;                  // floats per (species, x-box) intermediate block / per intermediate plane
    size_t smem;
    int threads, ctas_per_sm, grid;
};

// tallies of one context kept on the device
struct DevAcc {
    double released[2];
    double pad[6];
};

}  // namespace itk

struct it_ctx {
    itk::Grid g;
    double dx, dt;
    it_params p;
    int prec;             // IT_FP32 / IT_FP64
    size_t esize;         // element size
    void *n[2][2];        // [set][species]
    int cur;              // current set
    bool own_state;
    void *state_base;
    cudaStream_t stream;
    bool own_stream;
    int kernel;           // resolved IT_KERNEL_SIMPLE / IT_KERNEL_ZMARCH / IT_KERNEL_ZMARCH2
    int nslots;           // CTAs that own tally slots
    double *d_slots;      // [nslots][NT]
    double *d_mon;        // [nmon][NM]
    int nmon;
    double *d_acc;        // DevAcc
    double *d_out;        // finalize output [NT + NM + 2]
    double *h_out;        // pinned mirror
    // deposition scratch
    double *d_plane;      // [ny][nx] plane, then the per-tile sums of the deposit
    double *d_tracks;     // [cap][4]: x, y, LET, b
    double *d_angled;     // [angled_cap][5] tilted tracks (x, y, N0, b, theta), then per-block sums
    int64_t angled_cap;
    double *d_wx, *d_wy;  // [cap][nx], [cap][ny]
    int64_t track_cap;
    double *h_stage;      // pinned staging for host track uploads [stage_cap][4]
    int64_t stage_cap;
    cudaEvent_t stage_done;   // last upload from h_stage has completed
    // schedule (host, sorted by step)
    std::vector<int64_t> sched_step;
    std::vector<double> sched_tr;   // [n][4]
    size_t sched_ptr;
    int64_t steps;
    double t_s;                        // simulated time: the sum of every step's dt
    // time-step log: the first step of each dt, the dt and the peak density
    // that decided it (NaN for the initial dt)
    std::vector<int64_t> log_step;
    std::vector<double> log_dt, log_nmax;
    // graph of a fixed segment of steps
    cudaGraphExec_t graph;
    int graph_len;
    int graph_parity;
    // z-march kernel configuration (it_zmarch.cu)
    itk::ZmConf zm;
    int zm_grid;
    CUtensorMap tm_main[2][2];   // [set][species], box {bx, TY, 1} (4-D {256, nx/256, TY, 1} for nx > 256)
    CUtensorMap tm_halo[2][2];   // [set][species], box {bx, 1, 1} (4-D {256, nx/256, 1, 1} for nx > 256)
    itk::Zm2Conf zm2;            // two steps per launch (IT_KERNEL_ZMARCH2)
    CUtensorMap tm_main2[2][2];  // [set][species], box {bx, TY, 1}
    CUtensorMap tm_halo2[2][2];  // [set][species], box {bx, 2, 1}
    itk::Coef<float> cf;
    itk::Coef<double> cd;
    int *d_err;           // device error flag (bounded waits that ran out)
    long long wait_cycles;   // ring-wait limit of the z-march kernel (it_set_wait_limit)
    int withhold;            // test hook of it_test_withhold_load
};

namespace itk {

// thread-local error message
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define IT_CK(call)                                                  \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return itk::cuda_fail(_e, #call);     \
    } while (0)

// kernels (it_kernels.cu)
int launch_step_simple(it_ctx *c, cudaStream_t s);
int launch_step_zmarch(it_ctx *c, cudaStream_t s);
int zmarch_configure(it_ctx *c);
int zmarch_setup(it_ctx *c, int want_ty, int want_cps, int want_s, int want_grid);
// FP32 3-D tensor map over [nz][ny][nx] with a box of bx x rows x 1 (it_zmarch.cu)
int encode_map(CUtensorMap *m, void *base, int nx, int ny, int nz, int bx, int rows);
int encode_map_rows(CUtensorMap *m, void *base, int nx, int ny, int nz, int rows);
int encode_bf16_sw128(CUtensorMap *m, const void *base, long long K, long long rows, long long members,
                      long long row_bytes, long long member_bytes);
// two steps per launch (it_zmarch2.cu)
int zmarch2_setup(it_ctx *c, int want_ty, int want_cps, int want_s, int want_grid);
int launch_step_zmarch2(it_ctx *c, cudaStream_t s);
int set_launch(it_ctx *c, int kernel, int tile_rows, int ctas_per_sm, int stages, int grid);
int launch_finalize(it_ctx *c, cudaStream_t s);
int launch_monitor(it_ctx *c, cudaStream_t s);
int launch_deposit(it_ctx *c, int64_t n, cudaStream_t s);   // tracks already in d_tracks
int launch_zero(void *p, size_t bytes, cudaStream_t s);
int launch_deposit_angled(it_ctx *c, const double *d_tr, int64_t n, double *d_part, int nblocks, cudaStream_t s);
int simple_grid(const it_ctx *c);
int launch_step_simple_raw_f32(const float *ip, const float *im, float *op, float *om, int nx, int ny, int nz,
                               const Coef<float> &cf, bool periodic, double *slots, int nblocks, cudaStream_t s);
int launch_monitor_raw_f32(const float *p, const float *m, size_t cells, double vol, double *mon, int nblocks,
                           cudaStream_t s);
int validate_step_args(const it_params *p, it_grid g, double dx, double dt);
void coef_f32(const it_params *p, double dx, double dt, Coef<float> *out);
double ladder_rung(const it_params *p, double dx, double dt, double nmax);

}  // namespace itk
