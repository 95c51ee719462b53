/*
 * iontracks.h -- C ABI of the GB300 IonTracks transport library.
 *
 * The library evolves the positive and negative charge-carrier densities n+
 * and n- of an ionization chamber between two parallel electrodes
 * (Christensen, Toelli, Bassler, arXiv:1610.06749, Sec. "Charge carrier
 * movements", Eq. theEquation without the space-charge term):
 *
 *   dn+/dt = D+ lap n+ - mu+ E dn+/dz - alpha n+ n-
 *   dn-/dt = D- lap n- + mu- E dn-/dz - alpha n+ n-
 *
 * with the explicit scheme of the Appendix (forward Euler in time, the
 * blended backward/central drift derivative, which is Lax-Wendroff, and the
 * 3-point Laplacian), the time step bounded by Eq. (vNeum), Dirichlet
 * electrodes (Sec. Methods), Gaussian track deposition (Eqs. linear_density,
 * Gaussian, created) and tallies of released, recombined and collected
 * charge that give f = N_collected / N_released (Eq. collection_efficiency).
 *
 * Conventions (every entry point):
 *   - Units are CGS: cm, s, V, ions/cm^3; LET in keV/um; W in eV.
 *   - Return 0 (IT_OK) on success or a negative IT_E* code; nothing throws or
 *     aborts across the ABI.  it_last_error() gives a message for the last
 *     failure on the calling thread.
 *   - Host arrays passed in are read before the call returns; the caller
 *     keeps ownership.  Device memory the library allocates is freed by
 *     it_destroy; memory handed in through it_create_ex is never freed.
 *   - Work is enqueued on the context's CUDA stream; calls that return host
 *     results (it_tallies, it_get_density) synchronise that stream.
 *   - Grid layout of a density field: [nz][ny][nx], x fastest, densities of
 *     cell (i,j,k) whose extent is [i dx,(i+1) dx) x [j dx,(j+1) dx) x
 *     [k dx,(k+1) dx); the anode is the face z = 0, the cathode z = nz dx.
 *   - The library holds no CPU fallback: without a CUDA device every call
 *     that needs one returns IT_ECUDA.
 */
#ifndef IONTRACKS_H
#define IONTRACKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define IT_OK        0
#define IT_EINVAL   -1   /* bad argument or inconsistent parameters */
#define IT_ENOMEM   -2   /* device or host allocation failed */
#define IT_ECUDA    -3   /* a CUDA call failed (message in it_last_error) */
#define IT_EUNSTABLE -4  /* dt violates Eq. (vNeum) or the state went non-finite */
#define IT_ETIMEOUT -5   /* a bounded wait ran out */
#define IT_ESTATE   -6   /* call not valid in the context's current state */

/* it_params.precision: storage and update type of the densities; tallies are
 * always accumulated in FP64 */
#define IT_FP32 0
#define IT_FP64 1
/* it_params.lateral_bc: x/y faces.  The paper only asks that Lx, Ly be large
 * enough (Sec. Methods); periodic faces stand for a uniformly irradiated
 * chamber (Sec. Distribution of ion tracks), absorbing faces count what
 * leaves them in lost_lateral. */
#define IT_PERIODIC  0
#define IT_ABSORBING 1
/* it_params.scheme: drift derivative.  IT_LAX_WENDROFF is the Appendix's
 * blended derivative; IT_UPWIND the pure backward (upwind) difference. */
#define IT_LAX_WENDROFF 0
#define IT_UPWIND       1
/* it_params.kernel: which step kernel runs (all are CUDA). */
#define IT_KERNEL_AUTO   0   /* z-march kernel where the grid allows, else simple */
#define IT_KERNEL_SIMPLE 1   /* one thread per cell, global loads */
#define IT_KERNEL_ZMARCH 2   /* TMA-staged z-planes in shared memory (FP32, nx % 4 == 0) */
#define IT_KERNEL_ZMARCH2 3  /* as IT_KERNEL_ZMARCH, two time steps per launch (temporal blocking
                                of depth 2; nx/4 must divide 256 or 512 threads); densities are
                                bitwise those of two single steps */

typedef struct it_ctx it_ctx;

typedef struct {
    int32_t nx, ny, nz;     /* cells; gap = nz * dx */
} it_grid;

typedef struct {
    double mu[2];           /* mobilities [0] = positive, [1] = negative ions, cm^2/(V s) */
    double D[2];            /* diffusion constants, cm^2/s */
    double alpha;           /* recombination constant, cm^3/s */
    double W_eV;            /* mean energy per ion pair, eV (Eq. linear_density) */
    double gap_cm;          /* electrode gap d; must equal nz * dx (rel. 1e-9) */
    double voltage_V;       /* polarisation voltage; E = V / d along +z */
    int32_t precision;      /* IT_FP32 | IT_FP64 */
    int32_t lateral_bc;     /* IT_PERIODIC | IT_ABSORBING */
    int32_t scheme;         /* IT_LAX_WENDROFF | IT_UPWIND */
    int32_t kernel;         /* IT_KERNEL_* */
    double cfl_safety;      /* automatic dt = cfl_safety * dt_vN (default 1) */
    double react_kappa;     /* automatic dt <= react_kappa / (alpha n_peak) (default 0.5) */
    double n_peak_cm3;      /* peak density for that bound; 0 disables it */
    int32_t space_charge;   /* 1: include the space-charge term of Eq. (theEquation),
                               -/+ mu n div E with div E = q/eps0 (n+ - n-) (Maxwell-Gauss),
                               from the old level; the automatic dt then also satisfies
                               dt <= react_kappa / (max mu q/eps0 n_peak).  Default 0 */
    int32_t dt_ladder;      /* 1: it_run_to_completion raises dt at each check by the
                               doubling ladder (see there); 0: dt stays fixed.  Default 0 */
} it_params;

typedef struct {
    double released[2];          /* ions released per species (deposited in the domain) */
    double collected_anode[2];   /* ions that left through z = 0 (signed) */
    double collected_cathode[2]; /* ions that left through z = d (signed) */
    double lost_lateral[2];      /* ions that left through absorbing x/y faces */
    double in_domain[2];         /* ions still in the domain */
    double recombined;           /* ion pairs recombined */
    double f;                    /* (collected+ + collected-) / (released+ + released-) */
    double t_s;                  /* simulated time: the sum of every step's dt */
    double dt_s;                 /* time step */
    int64_t steps;               /* steps taken */
    double n_min[2], n_max[2];   /* extreme densities of the current state */
    double space_charge[2];      /* ions added to each species by the space-charge term
                                    (negative: removed; 0 when it is off).  The balance is
                                    released + space_charge = in_domain + collected
                                    + lost_lateral + recombined */
} it_tallies_t;

/* Library version string (static storage). */
const char *it_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *it_last_error(void);

/* Fill *p with the defaults: mu = 1.73 / 1.87, D = 0.037 / 0.037,
 * alpha = 1.6e-6, W = 34 eV, gap 0 (must be set), 0 V, FP32, periodic,
 * Lax-Wendroff, automatic kernel, cfl_safety 1, react_kappa 0.5, n_peak 0.
 * Returns IT_EINVAL if p is NULL. */
int it_params_default(it_params *p);

/* Largest time step allowed by Eq. (vNeum) for both species with E along z:
 * 2(sx+sy+sz) + cz^2 <= 1 (Lax-Wendroff) or 2(sx+sy+sz) + cz <= 1 (upwind),
 * s = D dt/dx^2, c = mu E dt/dx, times p->cfl_safety, and, when
 * p->n_peak_cm3 > 0 and alpha > 0, no larger than react_kappa/(alpha n_peak)
 * (the paper gives no bound for the reaction term; this keeps the explicit
 * recombination step monotone).  Writes the result to *dt_out. */
int it_auto_dt(const it_params *p, double dx_cm, double *dt_out);

/* Largest central density N0/(pi b^2), N0 = LET/W (Eqs. linear_density,
 * Gaussian) over n tracks; host arrays of n doubles.  For it_params.n_peak_cm3. */
int it_peak_density(int64_t n, const double *let_keV_um, const double *b_cm,
                    double W_eV, double *n_peak_out);

/* Bytes of device state a context of this grid and precision needs when the
 * caller provides it (it_create_ex): two ping-pong sets of both species. */
int it_state_bytes(it_grid g, int32_t precision, size_t *bytes_out);

/* Create a simulation with library-owned device memory on the current CUDA
 * device and a library-owned non-blocking stream.  dt_s <= 0 selects
 * it_auto_dt.  Densities start at zero.  Errors: IT_EINVAL (grid < 1 cell,
 * dx or constants non-positive or NaN, |gap - nz dx| > 1e-9 gap, dt above
 * the Eq. (vNeum) bound), IT_ENOMEM, IT_ECUDA. */
int it_create(it_grid g, double dx_cm, double dt_s, const it_params *p, it_ctx **out);

/* As it_create, but the density state lives in caller-owned device memory
 * dev_state of at least it_state_bytes() bytes (256-byte aligned), and work
 * is enqueued on the caller's stream (a cudaStream_t; NULL = a library
 * stream).  The library never frees dev_state or the stream. */
int it_create_ex(it_grid g, double dx_cm, double dt_s, const it_params *p,
                 void *dev_state, size_t bytes, void *stream, it_ctx **out);

/* Deposit n tracks parallel to the field now (instantaneous ionisation,
 * Sec. Implementation).  xy_cm: 2n doubles (x0,y0,x1,y1,...), let_keV_um and
 * b_cm: n doubles each, all host memory.  Each cell gains N0 wx wy / dx^2 on
 * every z plane for both species, wx = (erf((x_{i+1}-xc)/b) -
 * erf((x_i-xc)/b))/2 over a window of +-ceil(6 b/dx) cells around the centre
 * cell (wrapped when periodic, clipped when absorbing); released grows by what
 * landed in the domain.  n = 0 is a no-op.  Errors: IT_EINVAL for NULL arrays
 * with n > 0, b <= 0, LET < 0 or a non-finite value. */
int it_deposit_tracks(it_ctx *ctx, int64_t n, const double *xy_cm,
                      const double *let_keV_um, const double *b_cm);

/* Deposit n tracks at angles theta[i] in [0, pi/2] (radians) to the field
 * (Fig. setup (a)), each rotated in the x-z plane about an axis through
 * (xy_cm[2i], xy_cm[2i+1], d/2).  Eq. (Gaussian) about the axis: in the plane
 * of cell centres z_k the cross-section is a Gaussian of width b/cos(theta)
 * in x, centred at x + (z_k - d/2) tan(theta), and of width b in y; each cell
 * receives (N0/cos) wx wy / dx^2 with the cell-integrated weights wx, wy over
 * +-ceil(6 width/dx) cells (sampled at the cell centre in z).  Periodic faces
 * wrap the windows (the images of a tilted track are a periodic array of
 * parallel tracks); absorbing faces clip them.  Within cos(theta) dx/b < 1e-3
 * of parallel to the electrodes the track is a single column through the box,
 * each cell once, wx taken at the cell centre.  With periodic faces the two
 * descriptions differ at that switch by design: just outside it the images of
 * a track that crosses the gap over d tan(theta) in x stack up as many
 * parallel tracks; with absorbing faces the two forms agree there.  theta = 0 gives the densities
 * of it_deposit_tracks.  released grows by the FP64 sum deposited (N0 times
 * the path length when nothing is clipped).  One thread per cell visits
 * every track, so the cost is cells x n: for single tracks and small sets
 * (n <= 2^20).  Synchronous: returns after the deposit has run.  IT_EINVAL as
 * it_deposit_tracks, or for theta outside [0, pi/2] or NULL. */
int it_deposit_tracks_angled(it_ctx *ctx, int64_t n, const double *xy_cm, const double *let_keV_um,
                             const double *b_cm, const double *theta_rad);

/* As it_deposit_tracks, but the tracks are already in device memory as
 * n x 4 doubles (x_cm, y_cm, LET_keV_um, b_cm per track, 16-byte aligned),
 * enqueued on the context stream; nothing is validated on the host, so
 * values must be finite with b > 0.  For inputs kept resident in HBM. */
int it_deposit_tracks_device(it_ctx *ctx, int64_t n, const double *dev_tracks);

/* Schedule n tracks to be deposited at the start of step step_idx[i]
 * (counted from the context's step 0; Poisson-timed arrivals of a continuous
 * beam, Sec. Distribution of ion tracks).  Steps already taken are rejected
 * with IT_EINVAL.  Arrays as in it_deposit_tracks plus n int64 step indices.
 * Replaces any earlier schedule. */
int it_schedule_tracks(it_ctx *ctx, int64_t n, const double *xy_cm,
                       const double *let_keV_um, const double *b_cm,
                       const int64_t *step_idx);

/* Advance n_steps explicit steps (scheduled tracks deposited first at their
 * steps).  Asynchronous on the context stream; launches are replayed from a
 * captured CUDA graph in segments.  n_steps < 0 is IT_EINVAL. */
int it_step(it_ctx *ctx, int64_t n_steps);

/* Step until (in_domain+ + in_domain-) / (released+ + released-) < tol
 * ("dragged completely apart", Sec. Implementation), checked every
 * check_every steps, or until max_steps more steps.  *steps_done (may be NULL)
 * receives the steps taken.  Returns IT_EUNSTABLE if the state went
 * non-finite, IT_ETIMEOUT if max_steps ran out first.
 *
 * With params.dt_ladder = 1 and no scheduled tracks still to come, each check
 * that does not end the run first raises dt to min(cap, dt 2^j), j >= 0 the
 * largest integer with alpha (dt 2^j) n_max <= react_kappa (with the
 * space-charge term also max(mu) q/eps0 (dt 2^j) n_max <= react_kappa), where
 * n_max is the larger species maximum of the current state and cap is
 * cfl_safety times the Eq. (vNeum) step.  The recombination bound of
 * it_auto_dt is set by the densest cells, which recombine first; the ladder
 * applies the same bound to the state as it thins out, and never lowers dt.
 * Each change is logged (it_dt_log); the weights are rebuilt and the graph
 * segment recaptured. */
int it_run_to_completion(it_ctx *ctx, double tol, int64_t max_steps,
                         int64_t check_every, int64_t *steps_done);

/* Result of it_run_to_steady_state. */
typedef struct {
    double f_ss;          /* departure efficiency of every ion that left the domain since the
                             call began: Col / (Col + 2 Rec + Lost) over both species */
    double f_ss_stderr;   /* its standard error: the ratio estimator over 10 batches of
                             consecutive windows (NaN below 10 windows); batches shorter than
                             an ion's transit underestimate it */
    double f_window;      /* the last window's own departure efficiency (NaN: nothing left) */
    double departed;      /* ions that left the domain since the call began (Col + 2 Rec + Lost) */
    double released;      /* ions released since the call began */
    int64_t windows;      /* windows run */
    int64_t steps;        /* steps taken */
    int32_t stop;         /* 0: the steady-state rule ended the run; 1: the step limit did */
    int32_t pad_;
} it_steady_t;

/* Continuous beam run to steady state (Poisson arrivals scheduled with
 * it_schedule_tracks; Sec. Implementation, "Distribution of ion tracks"):
 * step in windows of window_steps, the caller having run any warm-up
 * before the call.  The cumulative f of it_tallies carries the ions still
 * in flight, so the rule judges the ions that have left the domain since
 * the call began: the aggregate f_ss = Col / (Col + 2 Rec + Lost), Col the
 * ions collected at either electrode, Rec the recombined pairs (two ions
 * each), Lost the ions lost through absorbing lateral faces.  The run stops
 * at the end of the first window, from the second on, after which f_ss has
 * moved by less than tol over that window ("f stable to tol over
 * window_steps steps"), provided the window carried departures of at least
 * half the mean release per window since the call began and the aggregate
 * covers at least half of the ions released since then (an idle window of
 * a sparse beam does not move f_ss and must not end the run); or when the
 * next whole window would pass max_steps more steps.  The run's precision
 * is f_ss_stderr, not tol.  *out (may be NULL) receives the result.
 * Returns IT_EUNSTABLE if the state went non-finite; reaching the step
 * limit is not an error. */
int it_run_to_steady_state(it_ctx *ctx, int64_t window_steps, double tol, int64_t max_steps,
                           it_steady_t *out);

/* Synchronise and return all tallies (FP64, reduced in a fixed order so that
 * reruns are bitwise identical). */
int it_tallies(it_ctx *ctx, it_tallies_t *out);

/* Copy one species' densities (0 = n+, 1 = n-) to host memory, [nz][ny][nx]
 * in the context's precision (bytes must equal cells * element size). */
int it_get_density(it_ctx *ctx, int species, void *host_dst, size_t bytes);

/* Replace both species' densities with host arrays (context precision,
 * [nz][ny][nx]) as an initial condition: all tallies restart, released
 * becomes the FP64 sum of what was set, the step counter and time return to
 * 0 and the time-step log restarts. */
int it_set_density(it_ctx *ctx, const void *plus, const void *minus, size_t bytes);

/* Set the time step before the first step (IT_ESTATE otherwise).  dt_s > 0
 * is checked against Eq. (vNeum); dt_s <= 0 applies it_auto_dt with n_peak
 * taken as the largest density of the current state (the deposited pulse,
 * overlaps of tracks included).  The recombination bound then holds for the
 * state actually deposited.  The time-step log restarts from the new dt. */
int it_retime(it_ctx *ctx, double dt_s);

/* One check of the dt ladder of it_run_to_completion, on the host: the dt
 * that a check with peak density n_max (ions/cm^3) picks after dt_s, for a
 * grid of spacing dx_cm under *p (gap_cm and voltage_V set the field).
 * *dt_out = min(cap, dt_s 2^j), j >= 0 the largest integer with
 * alpha (dt_s 2^j) n_max <= react_kappa (and, with space charge,
 * max(mu) q/eps0 (dt_s 2^j) n_max <= react_kappa); never below dt_s; cap =
 * cfl_safety times the Eq. (vNeum) step.  No device is needed.  IT_EINVAL for
 * NULL pointers, dx_cm or gap_cm <= 0, dt_s <= 0 or a negative or non-finite
 * n_max. */
int it_ladder_dt(const it_params *p, double dx_cm, double dt_s, double n_max, double *dt_out);

/* The time-step log: entry q holds the first step run with a dt
 * (first_step[q]), that dt (dt[q], s) and the peak density that decided it
 * (n_max[q], ions/cm^3; NaN for a dt set at creation, it_retime, it_reset or
 * it_set_density).  Entry 0 is the dt in force at step 0; it_run_to_completion
 * with the ladder appends one entry per rise.  Up to cap entries are written
 * to the caller's arrays (which may be NULL when cap is 0); *count receives
 * the number of entries in the log. */
int it_dt_log(it_ctx *ctx, int64_t cap, int64_t *first_step, double *dt, double *n_max, int64_t *count);

/* Return the context to its freshly created state without reallocating:
 * densities zero, all tallies zero, the device error flag cleared (after
 * IT_ETIMEOUT the context is usable again), step counter and time 0,
 * schedule cleared; the current dt stays and the time-step log restarts from
 * it.  Asynchronous on the context stream (no host synchronisation). */
int it_reset(it_ctx *ctx);

/* Device pointers of the current n+ and n- fields (valid until the next
 * it_step) and the context's stream (a cudaStream_t). */
int it_device_state(it_ctx *ctx, void **plus, void **minus, void **stream);

/* Choose the step kernel and, for IT_KERNEL_ZMARCH / IT_KERNEL_ZMARCH2, its
 * launch shape: rows per tile (a divisor of ny; for IT_KERNEL_ZMARCH2 it is
 * fixed at threads / (nx/4), 0 or that value), resident CTAs per SM (1: 16
 * warps, 2: 8 warps each) and ring depth (3..16); 0 leaves a value to the
 * built-in rule.  With IT_KERNEL_ZMARCH2, it_step runs steps in pairs and an
 * odd last step on the simple kernel.  Only before the first step (IT_ESTATE
 * otherwise).  IT_EINVAL if the shape does not fit the grid. */
int it_set_launch(it_ctx *ctx, int kernel, int tile_rows, int ctas_per_sm, int stages);

/* As it_set_launch, plus the grid of the z-march kernel: 0 = one CTA per
 * resident slot (SMs x ctas_per_sm); -1 = the largest multiple of the
 * y-tile count that fits those slots (every tile column is then cut at the
 * same z, so adjacent tiles are streamed in step); > 0 = that many CTAs. */
int it_set_launch_ex(it_ctx *ctx, int kernel, int tile_rows, int ctas_per_sm, int stages, int grid);

/* Time candidate launch shapes of the step kernel on the context's current
 * densities and keep the fastest (a native autotuner).  Each candidate runs
 * 2 untimed and trial_steps timed steps (rounded up to even, 8 if <= 0) on a
 * copy of the state, which is restored afterwards: the densities, tallies
 * and step counter are unchanged on return.  Only before the first step
 * (IT_ESTATE otherwise).  The choice is cached per grid shape, precision and
 * lateral boundary for the life of the process (flags & 1 forces a new
 * search).  *best_us (may be NULL) receives the chosen shape's time per
 * step in microseconds. */
int it_autotune(it_ctx *ctx, int trial_steps, int flags, double *best_us);

/* Report the kernel in use, its launch shape and its CTA count (for
 * IT_KERNEL_ZMARCH2, the CTAs of its two-step launches). */
int it_get_launch(it_ctx *ctx, int *kernel, int *tile_rows, int *ctas_per_sm, int *stages, int *ctas);

/* ---------------------------------------------------------------------------
 * Batched simulations: many independent simulations of uneven grids, each
 * with its own dx, voltage and time step, advanced together -- one launch
 * per step covers every simulation still running, and segments of launches
 * are replayed from a CUDA graph.  Each simulation computes exactly what a
 * single context with the same parameters computes (bitwise-identical
 * densities).
 * ------------------------------------------------------------------------- */
typedef struct it_batch it_batch;

typedef struct {
    int32_t nx, ny, nz;     /* cells; gap = nz * dx */
    double dx_cm;
    double dt_s;            /* <= 0: it_auto_dt with this simulation's voltage and n_peak */
    double voltage_V;
    double n_peak_cm3;      /* peak density for the recombination dt bound (0: none) */
} it_sim_desc;

/* Create nsim simulations.  common supplies mu, D, alpha, W, lateral_bc,
 * scheme, cfl_safety and react_kappa (its gap, voltage and n_peak are
 * ignored); precision must be IT_FP32.  Errors as for it_create, with the
 * offending simulation's index in the message. */
int it_batch_create(int32_t nsim, const it_sim_desc *descs, const it_params *common, it_batch **out);

/* Deposit n tracks into simulation `sim` (arrays as in it_deposit_tracks);
 * only before the first step (IT_ESTATE otherwise).  Synchronous. */
int it_batch_deposit_tracks(it_batch *b, int32_t sim, int64_t n, const double *xy_cm,
                            const double *let_keV_um, const double *b_cm);

/* Make simulation `sim` a train of `count` identical pulses: the tracks
 * deposited with it_batch_deposit_tracks are deposited again at the start
 * of steps period_steps, 2 period_steps, ...  (period_steps must be a
 * multiple of the even check interval of it_batch_run).  Before the first
 * step only. */
int it_batch_set_pulses(it_batch *b, int32_t sim, int32_t count, int64_t period_steps);

/* After the deposits (and it_batch_set_pulses) and before the first step:
 * every simulation created with dt_s <= 0 gets it_auto_dt with n_peak = the
 * largest density of its deposited state times its pulse count (IT_ESTATE
 * after the first step). */
int it_batch_retime(it_batch *b);

/* Cells per work-table entry (one CTA each; default 16384). */
int it_batch_set_chunk(it_batch *b, int64_t cells_per_block);

/* Native autotuner of the batched launch shape: after the deposits (and
 * it_batch_retime), before the first step.  Times trial_steps (>= 2, rounded
 * up to even) batched steps of the deposited state for each candidate --
 * the TMA-staged kernel with one or two float4 per thread or the register
 * float4 kernel, times z splits aiming at 1..32 CTAs per SM, times 4096 /
 * 16384 / 65536 cells per scalar-kernel entry when a simulation runs on the
 * scalar kernel (nx % 4 != 0) -- with CUDA events on the batch
 * stream, restores the deposited state after every trial (it allocates a
 * temporary copy of one state set, freed before return), keeps the fastest
 * and stores its microseconds per step in *best_us (may be NULL).  No tally
 * changes.  IT_ESTATE after the first step.  The paper has no batching; the
 * shape only changes the work split, not any cell's arithmetic. */
int it_batch_autotune(it_batch *b, int32_t trial_steps, double *best_us);

/* Run every simulation until its in-domain charge / released < tol or it
 * has taken max_steps steps, checked every check_every steps (rounded up to
 * even).  *launches (may be NULL) receives the number of step launches.
 * With common->dt_ladder = 1 every check also applies the doubling ladder of
 * it_run_to_completion to each active simulation whose pulses have all been
 * deposited (its own dx, voltage and peak density), so a simulation run in
 * the batch takes the same time steps as in its own context. */
int it_batch_run(it_batch *b, double tol, int64_t max_steps, int64_t check_every, int64_t *launches);

/* Tallies of one simulation (FP64; as it_tallies). */
int it_batch_tallies(it_batch *b, int32_t sim, it_tallies_t *out);

/* Densities of one simulation to host memory (FP32, [nz][ny][nx]). */
int it_batch_get_density(it_batch *b, int32_t sim, int species, void *host_dst, size_t bytes);

/* Free a batch; NULL is a no-op. */
int it_batch_destroy(it_batch *b);

/* ---------------------------------------------------------------------------
 * Surrogate network for f: an ensemble of perceptrons 6 -> 256 -> 256 ->
 * 256 -> 256 -> 1 (SiLU hidden layers, sigmoid output) trained by mean
 * squared error with Adam on solver results.  bfloat16 weights in the
 * matrix products, FP32 accumulation on the tensor cores, FP32 master
 * weights; reductions in a fixed order.  Inputs per sample: a row of 6
 * doubles describing a configuration (the surrogate workload uses log10 of
 * LET, voltage, gap, b, tracks per pulse and pulse period + 1 us); they are
 * normalised with the mean/std given to (or fitted by) the network.  The paper has no
 * counterpart: the surrogate answers f quickly and hands a configuration
 * back to the solver when its members disagree.
 * Parameter layout per member (floats): W1 [256][6], b1 [256], W2
 * [256][256], b2, W3, b3, W4, b4, W5 [1][256], b5 [1].
 * ------------------------------------------------------------------------- */
#define IT_MLP_INPUTS 6
#define IT_MLP_HIDDEN 256
#define IT_MLP_PARAMS 199425

typedef struct it_mlp it_mlp;

/* Create an ensemble of `members` networks (weights zero until set) with
 * work space for batches of up to max_batch samples. */
int it_mlp_create(int32_t members, int32_t max_batch, it_mlp **out);
/* Set / read one member's FP32 master parameters (count = IT_MLP_PARAMS);
 * setting restarts the optimiser state. */
int it_mlp_set_params(it_mlp *net, int32_t member, const float *params, int64_t count);
int it_mlp_get_params(it_mlp *net, int32_t member, float *out, int64_t count);
/* Input normalisation x' = (x - mean) / std (6 values each, std > 0), or
 * fitted to n samples. */
int it_mlp_set_normalization(it_mlp *net, const double *mean6, const double *std6);
int it_mlp_fit_normalization(it_mlp *net, int64_t n, const double *x);
/* Training set: n samples x (6 doubles), targets y (n doubles). */
int it_mlp_set_data(it_mlp *net, int64_t n, const double *x, const double *y);
/* `epochs` passes of Adam (beta 0.9 / 0.999, eps 1e-8, rate lr) over
 * mini-batches of `batch` samples in a SplitMix64 Fisher-Yates order from
 * `seed`, a different order for every member (ensemble diversity).  loss_per_epoch (may be NULL)
 * receives the mean over batches and members of the batch loss. */
int it_mlp_train(it_mlp *net, int32_t epochs, int32_t batch, double lr, uint64_t seed, double *loss_per_epoch);
/* Loss and gradient of every member on n <= max_batch samples (no update):
 * grads: members x IT_MLP_PARAMS floats, loss: members doubles.  The next
 * it_mlp_adam_step applies this gradient. */
int it_mlp_loss_grad(it_mlp *net, int64_t n, const double *x, const double *y, float *grads, double *loss);
int it_mlp_adam_step(it_mlp *net, double lr);
/* Predictions for n samples: ensemble mean and spread (max - min), and each
 * member's value (n x members, may be NULL). */
int it_mlp_predict(it_mlp *net, int64_t n, const double *x, double *mean, double *spread, double *per_member);
int it_mlp_destroy(it_mlp *net);

/* Capacity (CTAs) of the fixed tally scratch used by it_step_noalloc. */
#define IT_NOALLOC_MAX_BLOCKS 2048

/* One explicit step of both species without allocating device memory; the
 * paper has no counterpart -- this is for callers that may not call
 * cudaMalloc (code that only receives buffers from another framework's
 * memory pool, or a service that must not allocate after start-up).
 * dev_plus/dev_minus: this step's densities, dev_out_plus/dev_out_minus:
 * the next step's, FP32 [nz][ny][nx] device arrays that must not alias;
 * dev_tallies7: 7 device doubles that receive this step's recombined ion
 * pairs, anode +/-, cathode +/- and lateral +/- ions (the same quantities
 * it_tallies accumulates).  g, dx, dt and p as for it_create (p->precision
 * must be IT_FP32, p->space_charge 0; dt must be given and within Eq. (vNeum)).  Enqueued on
 * `stream` (a cudaStream_t, NULL = the legacy default stream).
 * The per-block tally partials live in one static device array of
 * IT_NOALLOC_MAX_BLOCKS x 10 doubles (160 KiB on each device that loads the
 * library, kept until exit); a device that would need more blocks is
 * rejected with IT_EINVAL.  The first call on a device looks up the array's
 * address (make it before any stream capture).  All calls share the array
 * and clear the part they use, so calls that overlap on the GPU race:
 * order them on one stream.  Allocates nothing: no cudaMalloc, cudaFree or
 * allocating library call. */
int it_step_noalloc(it_grid g, double dx_cm, double dt_s, const it_params *p,
                    const float *dev_plus, const float *dev_minus,
                    float *dev_out_plus, float *dev_out_minus,
                    double *dev_tallies7, void *stream);

/* How long (SM clock cycles) a ring wait of the z-march step kernel may
 * take before it is declared lost; 0 restores the default of 2^32 cycles
 * (about 2 s at 2 GHz).  A lost wait ends the launch early: the kernel waits
 * (always with the full 2^32-cycle bound) for the copies it has issued,
 * skips its tallies and raises the context's device error flag, which the
 * next it_tallies reports as IT_ETIMEOUT; it_reset clears it.  A caller
 * that must notice a stalled device quickly sets a shorter limit; a limit
 * shorter than a plane's load time makes normal steps fail.  The paper has
 * no counterpart.  IT_EINVAL for cycles < 0. */
int it_set_wait_limit(it_ctx *ctx, int64_t cycles);

/* Test hook for the bounded-wait path: with on = 1 the z-march kernel never
 * issues the first load of its plane ring, so the first wait of every warp
 * runs out after the it_set_wait_limit limit, without any fault: the
 * kernel drains the loads it did issue and returns, and IT_ETIMEOUT
 * follows as described there.  on = 0 restores normal steps.  IT_ESTATE if
 * the context does not run the z-march kernel (IT_KERNEL_ZMARCH). */
int it_test_withhold_load(it_ctx *ctx, int on);

/* Destroy a context; NULL is a no-op.  Synchronises the stream first. */
int it_destroy(it_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* IONTRACKS_H */
