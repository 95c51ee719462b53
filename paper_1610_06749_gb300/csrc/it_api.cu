// it_api.cu -- the C ABI (include/iontracks.h): parameters, time-step rule,
// context lifetime, deposition, stepping with CUDA-graph segments, tallies.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "it_internal.cuh"

namespace itk {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return IT_ECUDA;
}

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

// Eq. (vNeum) with E along z and dx = dy = dz: 6 s + c^2 <= 1 (Lax-Wendroff)
// or 6 s + c <= 1 (upwind), s = D dt/dx^2, c = mu E dt/dx.
// elementary charge (C) over the vacuum permittivity (F/cm), V cm
constexpr double kQOverEps0 = 1.602176634e-19 / 8.8541878128e-14;

static double dt_von_neumann(const it_params *p, double dx) {
    const double E = p->voltage_V / p->gap_cm;
    double best = INFINITY;
    for (int s = 0; s < 2; ++s) {
        const double q = 6.0 * p->D[s] / (dx * dx);
        const double v = p->mu[s] * E / dx;
        double dt;
        if (p->scheme == IT_UPWIND) {
            dt = (q + v) > 0 ? 1.0 / (q + v) : INFINITY;
        } else if (v > 0) {
            dt = (-q + std::sqrt(q * q + 4.0 * v * v)) / (2.0 * v * v);
        } else {
            dt = q > 0 ? 1.0 / q : INFINITY;
        }
        best = std::min(best, dt);
    }
    return best;
}

static int check_params(const it_params *p, it_grid g, double dx) {
    if (!p) return fail(IT_EINVAL, "params is NULL");
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(IT_EINVAL, "grid needs at least one cell per axis");
    if (!(std::isfinite(dx) && dx > 0)) return fail(IT_EINVAL, "dx must be positive and finite");
    for (int s = 0; s < 2; ++s)
        if (!finite_nonneg(p->mu[s]) || !finite_nonneg(p->D[s]))
            return fail(IT_EINVAL, "mobilities and diffusion constants must be finite and >= 0");
    if (!finite_nonneg(p->alpha) || !finite_nonneg(p->voltage_V))
        return fail(IT_EINVAL, "alpha and voltage must be finite and >= 0");
    if (!(std::isfinite(p->W_eV) && p->W_eV > 0)) return fail(IT_EINVAL, "W must be positive");
    if (!(std::isfinite(p->gap_cm) && p->gap_cm > 0)) return fail(IT_EINVAL, "gap must be positive");
    if (std::fabs(p->gap_cm - g.nz * dx) > 1e-9 * p->gap_cm)
        return fail(IT_EINVAL, "gap_cm must equal nz * dx");
    if (p->precision != IT_FP32 && p->precision != IT_FP64) return fail(IT_EINVAL, "bad precision");
    if (p->lateral_bc != IT_PERIODIC && p->lateral_bc != IT_ABSORBING) return fail(IT_EINVAL, "bad lateral_bc");
    if (p->scheme != IT_LAX_WENDROFF && p->scheme != IT_UPWIND) return fail(IT_EINVAL, "bad scheme");
    if (p->kernel < IT_KERNEL_AUTO || p->kernel > IT_KERNEL_ZMARCH2) return fail(IT_EINVAL, "bad kernel");
    if (!(std::isfinite(p->cfl_safety) && p->cfl_safety > 0 && p->cfl_safety <= 1.0))
        return fail(IT_EINVAL, "cfl_safety must be in (0, 1]");
    if (!(std::isfinite(p->react_kappa) && p->react_kappa > 0)) return fail(IT_EINVAL, "react_kappa must be > 0");
    if (!finite_nonneg(p->n_peak_cm3)) return fail(IT_EINVAL, "n_peak must be finite and >= 0");
    if (p->space_charge != 0 && p->space_charge != 1) return fail(IT_EINVAL, "space_charge must be 0 or 1");
    if (p->dt_ladder != 0 && p->dt_ladder != 1) return fail(IT_EINVAL, "dt_ladder must be 0 or 1");
    return IT_OK;
}

template <typename T>
static void make_coef(Coef<T> &cf, const it_params *p, double dx, double dt) {
    const double E = p->voltage_V / p->gap_cm;
    const double vol = dx * dx * dx;
    for (int s = 0; s < 2; ++s) {
        const double sigma = s == 0 ? 1.0 : -1.0;   // n+ drifts to +z, n- to -z
        const double c = p->mu[s] * E * dt / dx;
        const double sd = p->D[s] * dt / (dx * dx);
        double wzm, wzp;
        if (p->scheme == IT_UPWIND) {
            wzm = sd + (sigma > 0 ? c : 0.0);
            wzp = sd + (sigma > 0 ? 0.0 : c);
        } else {
            // Lax-Wendroff: n - (sigma c/2)(n_{k+1} - n_{k-1}) + (c^2/2)(n_{k+1} - 2n + n_{k-1})
            wzm = sd + 0.5 * c * c + 0.5 * sigma * c;
            wzp = sd + 0.5 * c * c - 0.5 * sigma * c;
        }
        // the update is an increment in flux form (upd7): each transport
        // weight multiplies a neighbour-minus-cell difference, so the
        // weights need no common rounding for charge to be conserved and
        // each is its own nearest value in T; wx = wy because the cells are
        // cubes, and the x and y terms share one weight in the update
        const double wx = sd, wy = sd;
        cf.wx[s] = (T)wx;
        cf.wy[s] = (T)wy;
        cf.wzm[s] = (T)wzm;
        cf.wzp[s] = (T)wzp;
        cf.anode_f[s] = (double)cf.wzp[s] * vol;
        cf.cathode_f[s] = (double)cf.wzm[s] * vol;
        cf.latx_f[s] = (double)cf.wx[s] * vol;
        cf.laty_f[s] = (double)cf.wy[s] * vol;
    }
    cf.adt = (T)(p->alpha * dt);
    cf.rec_f = (double)cf.adt * vol;
    // space charge, Eq. (theEquation): d n+/dt gains -mu+ n+ div E, d n-/dt gains
    // +mu- n- div E, div E = q/eps0 (n+ - n-)
    cf.sc_on = p->space_charge ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
        const double sigma = s == 0 ? 1.0 : -1.0;
        cf.sc[s] = p->space_charge ? (T)(-sigma * dt * p->mu[s] * kQOverEps0) : (T)0;
        cf.sc_f[s] = (double)cf.sc[s] * vol;
    }
}

static int ctx_free(it_ctx *c) {
    if (!c) return IT_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->own_state && c->state_base) cudaFree(c->state_base);
    cudaFree(c->d_slots);
    cudaFree(c->d_mon);
    cudaFree(c->d_acc);
    cudaFree(c->d_out);
    cudaFree(c->d_plane);
    cudaFree(c->d_tracks);
    cudaFree(c->d_angled);
    cudaFree(c->d_wx);
    cudaFree(c->d_wy);
    cudaFree(c->d_err);
    if (c->h_out) cudaFreeHost(c->h_out);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->stage_done) cudaEventDestroy(c->stage_done);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return IT_OK;
}

static int ensure_tracks(it_ctx *c, int64_t n) {
    if (n <= c->track_cap) return IT_OK;
    cudaFree(c->d_tracks); cudaFree(c->d_wx); cudaFree(c->d_wy);
    c->d_tracks = c->d_wx = c->d_wy = nullptr;
    c->track_cap = 0;
    IT_CK(cudaMalloc(&c->d_tracks, sizeof(double) * 4 * n));
    IT_CK(cudaMalloc(&c->d_wx, sizeof(double) * c->g.nx * n));
    IT_CK(cudaMalloc(&c->d_wy, sizeof(double) * c->g.ny * n));
    c->track_cap = n;
    return IT_OK;
}

constexpr int64_t kTrackChunk = 8192;

// pinned staging buffer for host track uploads; waits for the previous
// upload out of it before it is reused
static int stage_tracks(it_ctx *c, int64_t n, double **out) {
    if (c->stage_done) IT_CK(cudaEventSynchronize(c->stage_done));
    if (n > c->stage_cap) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->stage_cap = 0;
        IT_CK(cudaMallocHost(&c->h_stage, sizeof(double) * 4 * n));
        c->stage_cap = n;
    }
    if (!c->stage_done) IT_CK(cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming));
    *out = c->h_stage;
    return IT_OK;
}

// upload packed tracks [n][4] (pinned host memory) and deposit them, chunk by chunk
static int deposit_packed(it_ctx *c, const double *packed, int64_t n) {
    for (int64_t off = 0; off < n; off += kTrackChunk) {
        const int64_t m = std::min(kTrackChunk, n - off);
        int rc = ensure_tracks(c, m);
        if (rc) return rc;
        IT_CK(cudaMemcpyAsync(c->d_tracks, packed + 4 * off, sizeof(double) * 4 * m,
                              cudaMemcpyHostToDevice, c->stream));
        rc = launch_deposit(c, m, c->stream);
        if (rc) return rc;
    }
    if (n > 0 && c->stage_done) IT_CK(cudaEventRecord(c->stage_done, c->stream));
    return IT_OK;
}

static int validate_tracks(int64_t n, const double *xy, const double *let, const double *b) {
    if (n < 0) return fail(IT_EINVAL, "negative track count");
    if (n > 0 && (!xy || !let || !b)) return fail(IT_EINVAL, "track arrays are NULL");
    for (int64_t t = 0; t < n; ++t) {
        if (!std::isfinite(xy[2 * t]) || !std::isfinite(xy[2 * t + 1]))
            return fail(IT_EINVAL, "track position is not finite");
        if (!(std::isfinite(let[t]) && let[t] >= 0)) return fail(IT_EINVAL, "LET must be finite and >= 0");
        if (!(std::isfinite(b[t]) && b[t] > 0)) return fail(IT_EINVAL, "track radius b must be > 0");
    }
    return IT_OK;
}

static int one_step(it_ctx *c) {
    // the two-step kernel's odd steps run on the simple kernel (bitwise the same cells)
    return c->kernel == IT_KERNEL_ZMARCH ? launch_step_zmarch(c, c->stream) : launch_step_simple(c, c->stream);
}

// two steps: one launch of the two-step kernel, else two single steps
static int two_steps(it_ctx *c) {
    if (c->kernel == IT_KERNEL_ZMARCH2) return launch_step_zmarch2(c, c->stream);
    int rc = one_step(c);
    return rc ? rc : one_step(c);
}

constexpr int kGraphSteps = 32;   // even: a segment returns to the same ping-pong set

// run n steps with no deposit in between
static int run_plain(it_ctx *c, int64_t n) {
    while (n >= kGraphSteps) {
        if (!c->graph || c->graph_parity != c->cur) {
            if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
            const int start = c->cur;
            cudaGraph_t g = nullptr;
            IT_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            int rc = IT_OK;
            for (int q = 0; q < kGraphSteps && rc == IT_OK; q += 2) rc = two_steps(c);
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            c->cur = start;   // capture recorded the launches; nothing ran yet
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            c->graph_parity = start;
        }
        IT_CK(cudaGraphLaunch(c->graph, c->stream));
        n -= kGraphSteps;
        c->steps += kGraphSteps;
        c->t_s += c->dt * kGraphSteps;
    }
    for (; n >= 2; n -= 2) {
        int rc = two_steps(c);
        if (rc) return rc;
        c->steps += 2;
        c->t_s += c->dt * 2;
    }
    if (n == 1) {
        int rc = one_step(c);
        if (rc) return rc;
        c->steps += 1;
        c->t_s += c->dt;
    }
    return IT_OK;
}

// New time step for the steps that follow: weights, the log, and a new graph
// (a captured segment holds the old weights).
static void set_dt(it_ctx *c, double dt, double nmax) {
    c->dt = dt;
    make_coef(c->cf, &c->p, c->dx, dt);
    make_coef(c->cd, &c->p, c->dx, dt);
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    c->log_step.push_back(c->steps);
    c->log_dt.push_back(dt);
    c->log_nmax.push_back(nmax);
}

// One check of the doubling ladder: min(cap, dt 2^j) for the largest j >= 0
// with alpha (dt 2^j) n_max <= kappa (and, with space charge,
// max mu q/eps0 (dt 2^j) n_max <= kappa), never below dt.  cap is
// cfl_safety times the Eq. (vNeum) step.  Products are formed left to right.
double ladder_rung(const it_params *p, double dx, double dt, double nmax) {
    const double cap = p->cfl_safety * dt_von_neumann(p, dx);
    const double mu_max = std::max(p->mu[0], p->mu[1]);
    auto within = [&](double r) {
        if (p->alpha * r * nmax > p->react_kappa) return false;
        if (p->space_charge && mu_max * kQOverEps0 * r * nmax > p->react_kappa) return false;
        return true;
    };
    double r = dt;
    for (int q = 0; q < 60 && r < cap && within(2.0 * r); ++q) r *= 2.0;
    return std::max(dt, std::min(r, cap));
}

// Parameter and time-step checks of it_create, for entry points that take
// no context.
int validate_step_args(const it_params *p, it_grid g, double dx, double dt) {
    int rc = check_params(p, g, dx);
    if (rc) return rc;
    if (!(std::isfinite(dt) && dt > 0)) return fail(IT_EINVAL, "dt must be positive and finite");
    if (dt > dt_von_neumann(p, dx) * (1.0 + 1e-12)) return fail(IT_EINVAL, "dt exceeds the von Neumann bound of Eq. (vNeum)");
    return IT_OK;
}

void coef_f32(const it_params *p, double dx, double dt, Coef<float> *out) { make_coef(*out, p, dx, dt); }

// Reconfigure the step kernel (no step-count check); tally slots restart.
int set_launch(it_ctx *c, int kernel, int tile_rows, int ctas_per_sm, int stages, int grid) {
    if (kernel == IT_KERNEL_SIMPLE) {
        c->kernel = IT_KERNEL_SIMPLE;
    } else if (kernel == IT_KERNEL_ZMARCH2) {
        int rc = zmarch2_setup(c, tile_rows, ctas_per_sm, stages, grid);
        if (rc) return rc;
        c->kernel = IT_KERNEL_ZMARCH2;
    } else if (kernel == IT_KERNEL_ZMARCH || kernel == IT_KERNEL_AUTO) {
        int rc = zmarch_setup(c, tile_rows, ctas_per_sm, stages, grid);
        if (rc) {
            if (kernel == IT_KERNEL_ZMARCH) return rc;
            c->kernel = IT_KERNEL_SIMPLE;
        } else {
            c->kernel = IT_KERNEL_ZMARCH;
        }
    } else {
        return fail(IT_EINVAL, "bad kernel");
    }
    // the two-step kernel leaves odd steps to the simple kernel: slots for both
    const int n = c->kernel == IT_KERNEL_ZMARCH    ? c->zm_grid
                  : c->kernel == IT_KERNEL_ZMARCH2 ? std::max(c->zm2.grid, simple_grid(c))
                                                   : simple_grid(c);
    if (n != c->nslots) {
        double *ns = nullptr;
        IT_CK(cudaMalloc(&ns, sizeof(double) * NT * n));
        IT_CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->d_slots);
        c->d_slots = ns;
        c->nslots = n;
    }
    IT_CK(cudaMemsetAsync(c->d_slots, 0, sizeof(double) * NT * c->nslots, c->stream));
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return IT_OK;
}

}  // namespace itk

using namespace itk;

extern "C" {

const char *it_version(void) { return "iontracks-gb300 0.1 (sm_103a)"; }

const char *it_last_error(void) { return g_err.c_str(); }

int it_params_default(it_params *p) {
    if (!p) return fail(IT_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->mu[0] = 1.73; p->mu[1] = 1.87;
    p->D[0] = 0.037; p->D[1] = 0.037;
    p->alpha = 1.6e-6;
    p->W_eV = 34.0;
    p->precision = IT_FP32;
    p->lateral_bc = IT_PERIODIC;
    p->scheme = IT_LAX_WENDROFF;
    p->kernel = IT_KERNEL_AUTO;
    p->cfl_safety = 1.0;
    p->react_kappa = 0.5;
    return IT_OK;
}

int it_auto_dt(const it_params *p, double dx_cm, double *dt_out) {
    if (!p || !dt_out) return fail(IT_EINVAL, "NULL argument");
    if (!(std::isfinite(dx_cm) && dx_cm > 0) || !(p->gap_cm > 0)) return fail(IT_EINVAL, "dx and gap must be > 0");
    double dt = p->cfl_safety * dt_von_neumann(p, dx_cm);
    if (p->alpha > 0 && p->n_peak_cm3 > 0) dt = std::min(dt, p->react_kappa / (p->alpha * p->n_peak_cm3));
    // the space-charge term decays a lone species at the rate mu q/eps0 n
    if (p->space_charge && p->n_peak_cm3 > 0)
        dt = std::min(dt, p->react_kappa / (std::max(p->mu[0], p->mu[1]) * kQOverEps0 * p->n_peak_cm3));
    if (!std::isfinite(dt)) return fail(IT_EINVAL, "no finite time step (all transport constants are zero)");
    *dt_out = dt;
    return IT_OK;
}

int it_ladder_dt(const it_params *p, double dx_cm, double dt_s, double n_max, double *dt_out) {
    if (!p || !dt_out) return fail(IT_EINVAL, "NULL argument");
    if (!(std::isfinite(dx_cm) && dx_cm > 0) || !(p->gap_cm > 0)) return fail(IT_EINVAL, "dx and gap must be > 0");
    if (!(std::isfinite(dt_s) && dt_s > 0)) return fail(IT_EINVAL, "dt must be positive and finite");
    if (!(std::isfinite(n_max) && n_max >= 0)) return fail(IT_EINVAL, "n_max must be finite and >= 0");
    *dt_out = ladder_rung(p, dx_cm, dt_s, n_max);
    return IT_OK;
}

int it_peak_density(int64_t n, const double *let, const double *b, double W_eV, double *out) {
    if (!out || n < 0 || (n > 0 && (!let || !b)) || !(W_eV > 0)) return fail(IT_EINVAL, "bad argument");
    double best = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        const double N0 = let[t] * 1e7 / W_eV;
        best = std::max(best, N0 / (M_PI * b[t] * b[t]));
    }
    *out = best;
    return IT_OK;
}

int it_state_bytes(it_grid g, int32_t precision, size_t *bytes_out) {
    if (!bytes_out || g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(IT_EINVAL, "bad grid");
    const size_t es = precision == IT_FP64 ? 8 : 4;
    const size_t cells = (size_t)g.nx * g.ny * g.nz;
    // four arrays, each rounded up to 256 bytes
    const size_t one = (cells * es + 255) / 256 * 256;
    *bytes_out = 4 * one;
    return IT_OK;
}

int it_create_ex(it_grid g, double dx_cm, double dt_s, const it_params *p, void *dev_state, size_t bytes,
                 void *stream, it_ctx **out) {
    if (!out) return fail(IT_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(p, g, dx_cm);
    if (rc) return rc;
    double dtmax = 0.0;
    rc = it_auto_dt(p, dx_cm, &dtmax);
    if (rc) return rc;
    double dt = dt_s;
    if (!(dt_s > 0)) {
        dt = dtmax;
    } else {
        const double vn = dt_von_neumann(p, dx_cm);
        if (!std::isfinite(dt_s) || dt_s > vn * (1.0 + 1e-12))
            return fail(IT_EINVAL, "dt exceeds the von Neumann bound of Eq. (vNeum)");
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(IT_ECUDA, "no CUDA device available");

    it_ctx *c = new (std::nothrow) it_ctx();
    if (!c) return fail(IT_ENOMEM, "host allocation failed");
    c->g = Grid{g.nx, g.ny, g.nz};
    c->dx = dx_cm;
    c->dt = dt;
    c->p = *p;
    c->prec = p->precision;
    c->esize = p->precision == IT_FP64 ? 8 : 4;
    c->graph_parity = -1;
    c->log_step.assign(1, 0);
    c->log_dt.assign(1, dt);
    c->log_nmax.assign(1, std::nan(""));

    auto bail = [&](int code) { ctx_free(c); return code; };

    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
        c->own_stream = true;
    }
    size_t need = 0;
    it_state_bytes(g, p->precision, &need);
    const size_t one = need / 4;
    if (dev_state) {
        if (bytes < need) return bail(fail(IT_EINVAL, "dev_state smaller than it_state_bytes()"));
        if (((uintptr_t)dev_state & 255) != 0) return bail(fail(IT_EINVAL, "dev_state must be 256-byte aligned"));
        c->state_base = dev_state;
        c->own_state = false;
    } else {
        e = cudaMalloc(&c->state_base, need);
        if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? fail(IT_ENOMEM, "state allocation failed")
                                                                          : cuda_fail(e, "cudaMalloc"));
        c->own_state = true;
    }
    char *base = (char *)c->state_base;
    c->n[0][0] = base; c->n[0][1] = base + one; c->n[1][0] = base + 2 * one; c->n[1][1] = base + 3 * one;
    c->cur = 0;
    e = cudaMemsetAsync(c->state_base, 0, need, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemset"));

    make_coef(c->cf, p, dx_cm, dt);
    make_coef(c->cd, p, dx_cm, dt);

    // kernel choice
    c->kernel = IT_KERNEL_SIMPLE;
    if (p->kernel == IT_KERNEL_ZMARCH || p->kernel == IT_KERNEL_AUTO) {
        rc = zmarch_configure(c);
        if (rc == IT_OK) {
            c->kernel = IT_KERNEL_ZMARCH;
        } else if (p->kernel == IT_KERNEL_ZMARCH) {
            return bail(rc);
        }
    } else if (p->kernel == IT_KERNEL_ZMARCH2) {
        rc = zmarch2_setup(c, 0, 0, 0, 0);
        if (rc) return bail(rc);
        c->kernel = IT_KERNEL_ZMARCH2;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the two-step kernel leaves odd steps to the simple kernel: slots for both
    c->nslots = c->kernel == IT_KERNEL_ZMARCH    ? c->zm_grid
                : c->kernel == IT_KERNEL_ZMARCH2 ? std::max(c->zm2.grid, simple_grid(c))
                                                 : simple_grid(c);
    c->nmon = 2 * sms;

    if ((e = cudaMalloc(&c->d_slots, sizeof(double) * NT * c->nslots)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_mon, sizeof(double) * NM * c->nmon)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_acc, sizeof(DevAcc))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_out, sizeof(double) * NOUT)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_plane, sizeof(double) * 2 * c->g.plane())) != cudaSuccess ||   // plane + tile sums
        (e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_out, sizeof(double) * NOUT)) != cudaSuccess)
        return bail(cuda_fail(e, "scratch allocation"));
    if ((e = cudaMemsetAsync(c->d_slots, 0, sizeof(double) * NT * c->nslots, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_acc, 0, sizeof(DevAcc), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemset"));
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(e, "create sync"));
    *out = c;
    return IT_OK;
}

int it_create(it_grid g, double dx_cm, double dt_s, const it_params *p, it_ctx **out) {
    return it_create_ex(g, dx_cm, dt_s, p, nullptr, 0, nullptr, out);
}

int it_deposit_tracks(it_ctx *c, int64_t n, const double *xy, const double *let, const double *b) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    int rc = validate_tracks(n, xy, let, b);
    if (rc || n == 0) return rc;
    double *packed = nullptr;
    rc = stage_tracks(c, n, &packed);
    if (rc) return rc;
    for (int64_t t = 0; t < n; ++t) {
        packed[4 * t + 0] = xy[2 * t];
        packed[4 * t + 1] = xy[2 * t + 1];
        packed[4 * t + 2] = let[t];
        packed[4 * t + 3] = b[t];
    }
    return deposit_packed(c, packed, n);
}

int it_deposit_tracks_angled(it_ctx *c, int64_t n, const double *xy, const double *let, const double *b,
                             const double *theta) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    int rc = validate_tracks(n, xy, let, b);
    if (rc || n == 0) return rc;
    if (!theta) return fail(IT_EINVAL, "theta is NULL");
    for (int64_t t = 0; t < n; ++t)
        if (!(theta[t] >= 0.0 && theta[t] <= 1.5707963267948966))
            return fail(IT_EINVAL, "theta must lie in [0, pi/2]");
    if (n > (1 << 20)) return fail(IT_EINVAL, "at most 2^20 tilted tracks per call");
    // track records, then one FP64 partial sum per block of the kernel
    constexpr int kBlocks = 1216;   // 8 per SM on 152 SMs; fixed, so the sums are deterministic
    const int64_t need = 5 * n + kBlocks;
    if (need > c->angled_cap) {
        cudaFree(c->d_angled);
        c->d_angled = nullptr;
        c->angled_cap = 0;
        IT_CK(cudaMalloc(&c->d_angled, sizeof(double) * need));
        c->angled_cap = need;
    }
    std::vector<double> h((size_t)5 * n);
    for (int64_t t = 0; t < n; ++t) {
        h[5 * t + 0] = xy[2 * t];
        h[5 * t + 1] = xy[2 * t + 1];
        h[5 * t + 2] = let[t] * 1e7 / c->p.W_eV;   // Eq. (linear_density), ions/cm
        h[5 * t + 3] = b[t];
        h[5 * t + 4] = theta[t];
    }
    IT_CK(cudaMemcpyAsync(c->d_angled, h.data(), sizeof(double) * 5 * n, cudaMemcpyHostToDevice, c->stream));
    rc = launch_deposit_angled(c, c->d_angled, n, c->d_angled + 5 * n, kBlocks, c->stream);
    if (rc) return rc;
    IT_CK(cudaStreamSynchronize(c->stream));   // the host records are released on return
    return IT_OK;
}

int it_deposit_tracks_device(it_ctx *c, int64_t n, const double *dev_tracks) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (n < 0 || (n > 0 && !dev_tracks)) return fail(IT_EINVAL, "bad track array");
    for (int64_t off = 0; off < n; off += kTrackChunk) {
        const int64_t m = std::min(kTrackChunk, n - off);
        int rc = ensure_tracks(c, m);
        if (rc) return rc;
        IT_CK(cudaMemcpyAsync(c->d_tracks, dev_tracks + 4 * off, sizeof(double) * 4 * m, cudaMemcpyDeviceToDevice,
                              c->stream));
        rc = launch_deposit(c, m, c->stream);
        if (rc) return rc;
    }
    return IT_OK;
}

int it_schedule_tracks(it_ctx *c, int64_t n, const double *xy, const double *let, const double *b,
                       const int64_t *step_idx) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    int rc = validate_tracks(n, xy, let, b);
    if (rc) return rc;
    if (n > 0 && !step_idx) return fail(IT_EINVAL, "step_idx is NULL");
    for (int64_t t = 0; t < n; ++t)
        if (step_idx[t] < c->steps) return fail(IT_EINVAL, "a scheduled step has already been taken");
    std::vector<int64_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t bb) { return step_idx[a] < step_idx[bb]; });
    c->sched_step.resize((size_t)n);
    c->sched_tr.resize((size_t)n * 4);
    for (int64_t q = 0; q < n; ++q) {
        const int64_t t = order[q];
        c->sched_step[q] = step_idx[t];
        c->sched_tr[4 * q + 0] = xy[2 * t];
        c->sched_tr[4 * q + 1] = xy[2 * t + 1];
        c->sched_tr[4 * q + 2] = let[t];
        c->sched_tr[4 * q + 3] = b[t];
    }
    c->sched_ptr = 0;
    return IT_OK;
}

int it_step(it_ctx *c, int64_t n) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (n < 0) return fail(IT_EINVAL, "negative step count");
    const int64_t end = c->steps + n;
    while (c->steps < end) {
        // deposit tracks that arrive at the start of this step
        size_t q = c->sched_ptr;
        while (q < c->sched_step.size() && c->sched_step[q] == c->steps) ++q;
        if (q > c->sched_ptr) {
            const int64_t m = (int64_t)(q - c->sched_ptr);
            double *packed = nullptr;
            int rc = stage_tracks(c, m, &packed);
            if (rc) return rc;
            std::memcpy(packed, c->sched_tr.data() + 4 * c->sched_ptr, sizeof(double) * 4 * m);
            rc = deposit_packed(c, packed, m);
            if (rc) return rc;
            c->sched_ptr = q;
        }
        int64_t until = end;
        if (c->sched_ptr < c->sched_step.size()) until = std::min(until, c->sched_step[c->sched_ptr]);
        if (until <= c->steps) until = c->steps + 1;
        int rc = run_plain(c, until - c->steps);
        if (rc) return rc;
    }
    return IT_OK;
}

int it_tallies(it_ctx *c, it_tallies_t *t) {
    if (!c || !t) return fail(IT_EINVAL, "NULL argument");
    int rc = launch_monitor(c, c->stream);
    if (rc) return rc;
    rc = launch_finalize(c, c->stream);
    if (rc) return rc;
    IT_CK(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * NOUT, cudaMemcpyDeviceToHost, c->stream));
    IT_CK(cudaStreamSynchronize(c->stream));
    const double *o = c->h_out;
    std::memset(t, 0, sizeof(*t));
    t->recombined = o[0];
    t->collected_anode[0] = o[1]; t->collected_anode[1] = o[2];
    t->collected_cathode[0] = o[3]; t->collected_cathode[1] = o[4];
    t->lost_lateral[0] = o[5]; t->lost_lateral[1] = o[6];
    t->space_charge[0] = o[7]; t->space_charge[1] = o[8];
    t->in_domain[0] = o[NT]; t->in_domain[1] = o[NT + 1];
    t->n_min[0] = o[NT + 2]; t->n_min[1] = o[NT + 3];
    t->n_max[0] = o[NT + 4]; t->n_max[1] = o[NT + 5];
    t->released[0] = o[NT + NM]; t->released[1] = o[NT + NM + 1];
    const double rel = t->released[0] + t->released[1];
    const double col = t->collected_anode[0] + t->collected_anode[1] + t->collected_cathode[0] + t->collected_cathode[1];
    t->f = rel > 0 ? col / rel : NAN;
    t->steps = c->steps;
    t->dt_s = c->dt;
    t->t_s = c->t_s;
    if (o[NT + NM + 2] != 0.0) return fail(IT_ETIMEOUT, "a bounded device wait ran out in the step kernel");
    return IT_OK;
}

int it_run_to_completion(it_ctx *c, double tol, int64_t max_steps, int64_t check_every, int64_t *steps_done) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (!(tol >= 0) || max_steps < 0 || check_every < 1) return fail(IT_EINVAL, "bad argument");
    const int64_t start = c->steps;
    it_tallies_t t;
    int rc = IT_OK;
    for (;;) {
        rc = it_tallies(c, &t);
        if (rc) break;
        if (!std::isfinite(t.in_domain[0] + t.in_domain[1] + t.recombined)) { rc = fail(IT_EUNSTABLE, "state is not finite"); break; }
        const double rel = t.released[0] + t.released[1];
        // scheduled tracks still to come keep the run going
        const bool pending = c->sched_ptr < c->sched_step.size();
        if (!pending && rel > 0 && (t.in_domain[0] + t.in_domain[1]) / rel < tol) break;
        if (!pending && rel == 0) break;
        const int64_t left = start + max_steps - c->steps;
        if (left <= 0) { rc = fail(IT_ETIMEOUT, "max_steps reached before completion"); break; }
        // the ladder: only while no scheduled deposit can raise the densities
        if (c->p.dt_ladder && !pending) {
            const double nmax = std::max(t.n_max[0], t.n_max[1]);
            const double nd = ladder_rung(&c->p, c->dx, c->dt, nmax);
            if (nd > c->dt) set_dt(c, nd, nmax);
        }
        rc = it_step(c, std::min(check_every, left));
        if (rc) break;
    }
    if (steps_done) *steps_done = c->steps - start;
    return rc;
}

int it_run_to_steady_state(it_ctx *c, int64_t window_steps, double tol, int64_t max_steps, it_steady_t *out) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (window_steps < 1 || !(tol >= 0) || max_steps < 0) return fail(IT_EINVAL, "bad argument");
    const int64_t start = c->steps;
    it_tallies_t t;
    int rc = it_tallies(c, &t);
    // ions that have left the domain so far, by route, and ions released
    auto col = [](const it_tallies_t &x) {
        return x.collected_anode[0] + x.collected_anode[1] + x.collected_cathode[0] + x.collected_cathode[1];
    };
    auto lost = [](const it_tallies_t &x) { return x.lost_lateral[0] + x.lost_lateral[1]; };
    auto rel = [](const it_tallies_t &x) { return x.released[0] + x.released[1]; };
    const double c_start = col(t), r_start = t.recombined, l_start = lost(t), rel_start = rel(t);
    double c0 = c_start, r0 = r_start, l0 = l_start;
    // per-window collected and departed ions, for the batch-means error
    std::vector<double> wc, wg;
    double F_prev = std::nan(""), F = std::nan(""), f_win = std::nan("");
    double C = 0.0, G = 0.0, Rel = 0.0;
    int code = 1;
    while (rc == IT_OK && c->steps - start + window_steps <= max_steps) {
        rc = it_step(c, window_steps);
        if (rc) break;
        rc = it_tallies(c, &t);
        if (rc) break;
        if (!std::isfinite(t.in_domain[0] + t.in_domain[1] + t.recombined)) { rc = fail(IT_EUNSTABLE, "state is not finite"); break; }
        const double dc = col(t) - c0, dr = t.recombined - r0, dl = lost(t) - l0;
        c0 = col(t); r0 = t.recombined; l0 = lost(t);
        const double g = dc + 2.0 * dr + dl;   // a recombined pair removes two ions
        wc.push_back(dc);
        wg.push_back(g);
        f_win = g != 0.0 ? dc / g : std::nan("");
        // aggregate since the call began (sums of the cumulative tallies'
        // differences, so no window's rounding is lost)
        C = col(t) - c_start;
        G = C + 2.0 * (t.recombined - r_start) + (lost(t) - l_start);
        Rel = rel(t) - rel_start;
        F = G != 0.0 ? C / G : std::nan("");
        const double n = (double)wc.size();
        // a window is judged only when it carried departures of at least half
        // the mean release per window, and the aggregate at least half of
        // everything released since the call began
        const bool judged = g > 0.0 && g >= 0.5 * Rel / n && G >= 0.5 * Rel;
        if (judged && wc.size() >= 2 && std::isfinite(F) && std::isfinite(F_prev) && std::fabs(F - F_prev) < tol) {
            code = 0;
            break;
        }
        F_prev = F;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->f_ss = F;
        out->f_window = f_win;
        out->departed = G;
        out->released = Rel;
        out->windows = (int64_t)wc.size();
        out->steps = c->steps - start;
        out->stop = code;
        // ratio estimator C/G with batch means over nb contiguous batches of windows
        const int64_t n = (int64_t)wc.size();
        const int64_t nb = n >= 10 ? 10 : 0;
        double se = std::nan("");
        if (nb >= 2 && G != 0.0 && std::isfinite(F)) {
            double ss = 0.0;
            for (int64_t b = 0; b < nb; ++b) {
                double cb = 0.0, gb = 0.0;
                for (int64_t w = b * n / nb; w < (b + 1) * n / nb; ++w) { cb += wc[w]; gb += wg[w]; }
                const double e = cb - F * gb;
                ss += e * e;
            }
            se = std::sqrt(ss * (double)nb / (double)(nb - 1)) / G;
        }
        out->f_ss_stderr = se;
    }
    return rc;
}

int it_get_density(it_ctx *c, int species, void *dst, size_t bytes) {
    if (!c || !dst || (species != 0 && species != 1)) return fail(IT_EINVAL, "bad argument");
    if (bytes != c->g.cells() * c->esize) return fail(IT_EINVAL, "bytes must equal cells * element size");
    IT_CK(cudaMemcpyAsync(dst, c->n[c->cur][species], bytes, cudaMemcpyDeviceToHost, c->stream));
    IT_CK(cudaStreamSynchronize(c->stream));
    return IT_OK;
}

int it_set_density(it_ctx *c, const void *plus, const void *minus, size_t bytes) {
    if (!c || !plus || !minus) return fail(IT_EINVAL, "bad argument");
    if (bytes != c->g.cells() * c->esize) return fail(IT_EINVAL, "bytes must equal cells * element size");
    IT_CK(cudaMemcpyAsync(c->n[c->cur][0], plus, bytes, cudaMemcpyHostToDevice, c->stream));
    IT_CK(cudaMemcpyAsync(c->n[c->cur][1], minus, bytes, cudaMemcpyHostToDevice, c->stream));
    IT_CK(cudaMemsetAsync(c->d_slots, 0, sizeof(double) * NT * c->nslots, c->stream));
    IT_CK(cudaMemsetAsync(c->d_acc, 0, sizeof(DevAcc), c->stream));
    c->steps = 0;
    c->t_s = 0.0;
    c->sched_step.clear(); c->sched_tr.clear(); c->sched_ptr = 0;
    c->log_step.assign(1, 0);
    c->log_dt.assign(1, c->dt);
    c->log_nmax.assign(1, std::nan(""));
    it_tallies_t t;
    int rc = it_tallies(c, &t);
    if (rc) return rc;
    DevAcc a{};
    a.released[0] = t.in_domain[0];
    a.released[1] = t.in_domain[1];
    IT_CK(cudaMemcpyAsync(c->d_acc, &a, sizeof(a), cudaMemcpyHostToDevice, c->stream));
    IT_CK(cudaStreamSynchronize(c->stream));
    return IT_OK;
}

int it_retime(it_ctx *c, double dt_s) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (c->steps != 0) return fail(IT_ESTATE, "the time step can only change before the first step");
    it_params p = c->p;
    double dt = dt_s;
    if (!(dt_s > 0)) {
        it_tallies_t t;
        int rc = it_tallies(c, &t);
        if (rc) return rc;
        const double npk = std::max(t.n_max[0], t.n_max[1]);
        if (!std::isfinite(npk)) return fail(IT_EUNSTABLE, "state is not finite");
        p.n_peak_cm3 = npk > 0 ? npk : 0.0;
        rc = it_auto_dt(&p, c->dx, &dt);
        if (rc) return rc;
    } else if (!std::isfinite(dt_s) || dt_s > dt_von_neumann(&p, c->dx) * (1.0 + 1e-12)) {
        return fail(IT_EINVAL, "dt exceeds the von Neumann bound of Eq. (vNeum)");
    }
    c->p = p;
    c->log_step.clear(); c->log_dt.clear(); c->log_nmax.clear();
    set_dt(c, dt, std::nan(""));
    return IT_OK;
}

int it_reset(it_ctx *c) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    const size_t bytes = c->g.cells() * c->esize;
    IT_CK(cudaMemsetAsync(c->n[c->cur][0], 0, bytes, c->stream));
    IT_CK(cudaMemsetAsync(c->n[c->cur][1], 0, bytes, c->stream));
    IT_CK(cudaMemsetAsync(c->d_slots, 0, sizeof(double) * NT * c->nslots, c->stream));
    IT_CK(cudaMemsetAsync(c->d_acc, 0, sizeof(DevAcc), c->stream));
    IT_CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    c->steps = 0;
    c->t_s = 0.0;
    c->sched_step.clear(); c->sched_tr.clear(); c->sched_ptr = 0;
    // the time step stays; the log restarts from it
    c->log_step.assign(1, 0);
    c->log_dt.assign(1, c->dt);
    c->log_nmax.assign(1, std::nan(""));
    return IT_OK;
}

int it_dt_log(it_ctx *c, int64_t cap, int64_t *first_step, double *dt, double *n_max, int64_t *count) {
    if (!c || !count || cap < 0) return fail(IT_EINVAL, "bad argument");
    const int64_t n = (int64_t)c->log_step.size();
    const int64_t m = std::min(n, cap);
    if (m > 0 && (!first_step || !dt || !n_max)) return fail(IT_EINVAL, "NULL output array");
    for (int64_t q = 0; q < m; ++q) {
        first_step[q] = c->log_step[q];
        dt[q] = c->log_dt[q];
        n_max[q] = c->log_nmax[q];
    }
    *count = n;
    return IT_OK;
}

int it_device_state(it_ctx *c, void **plus, void **minus, void **stream) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (plus) *plus = c->n[c->cur][0];
    if (minus) *minus = c->n[c->cur][1];
    if (stream) *stream = (void *)c->stream;
    return IT_OK;
}

int it_set_launch_ex(it_ctx *c, int kernel, int tile_rows, int ctas_per_sm, int stages, int grid) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (c->steps != 0) return fail(IT_ESTATE, "launch shape can only change before the first step");
    return set_launch(c, kernel, tile_rows, ctas_per_sm, stages, grid);
}

int it_set_launch(it_ctx *c, int kernel, int tile_rows, int ctas_per_sm, int stages) {
    return it_set_launch_ex(c, kernel, tile_rows, ctas_per_sm, stages, 0);
}

int it_get_launch(it_ctx *c, int *kernel, int *tile_rows, int *ctas_per_sm, int *stages, int *ctas) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    const bool zm = c->kernel == IT_KERNEL_ZMARCH, zm2 = c->kernel == IT_KERNEL_ZMARCH2;
    if (kernel) *kernel = c->kernel;
    if (tile_rows) *tile_rows = zm ? c->zm.TY : zm2 ? c->zm2.TY : 0;
    if (ctas_per_sm) *ctas_per_sm = zm ? c->zm.ctas_per_sm : zm2 ? c->zm2.ctas_per_sm : 0;
    if (stages) *stages = zm ? c->zm.S : zm2 ? c->zm2.S : 0;
    if (ctas) *ctas = zm2 ? c->zm2.grid : c->nslots;
    return IT_OK;
}

int it_set_wait_limit(it_ctx *c, int64_t cycles) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (cycles < 0) return fail(IT_EINVAL, "cycles must be >= 0");
    c->wait_cycles = cycles;
    // a captured segment holds the old kernel arguments
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return IT_OK;
}

int it_test_withhold_load(it_ctx *c, int on) {
    if (!c) return fail(IT_EINVAL, "ctx is NULL");
    if (on != 0 && on != 1) return fail(IT_EINVAL, "on must be 0 or 1");
    if (on && c->kernel != IT_KERNEL_ZMARCH) return fail(IT_ESTATE, "the test hook applies to the z-march kernel only");
    c->withhold = on;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return IT_OK;
}

int it_destroy(it_ctx *c) { return ctx_free(c); }

}  // extern "C"
