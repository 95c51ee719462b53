/*
 * iontracks_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the discretised IonTracks equations
 * (Christensen, Toelli, Bassler, arXiv:1610.06749).  Only tests/, the smoke
 * check and the CPU-baseline leg of the benchmark may load this library; the
 * product path never does.  It shares no code, header, table or constant with
 * the CUDA library: everything here is written from the paper directly.
 *
 * What it computes, in the paper's order:
 *   - Deposition: linear density N0 = LET/W (Eq. linear_density) spread with
 *     Jaffe's Gaussian radial profile n0(r) = N0/(pi b^2) exp(-r^2/b^2)
 *     (Eq. Gaussian), integrated over each cell (cell-average reading), for a
 *     track parallel to the field that spans the gap, so the released charge is
 *     N0 * l (Eq. created) minus whatever falls outside an absorbing domain.
 *   - Transport: the continuity equations of Eq. (cont_eq)/(theEquation) with a
 *     uniform external field E = V/d along +z, discretised as in
 *     the Appendix: forward-Euler time derivative, the blended
 *     backward/central first derivative weighted by c = mu E dt/dz, and the
 *     3-point second derivative per axis.  The upwind side follows each
 *     species' own drift direction (reading).  Recombination -alpha n+ n- is
 *     taken from the old time level.
 *   - Space charge (optional, off by default): the term -/+ mu n div E of Eq.
 *     (theEquation) with div E from the Maxwell-Gauss equation,
 *     div E = q/eps0 (n+ - n-), also from the old time level; its net change
 *     of each species is tallied (the term as printed does not conserve
 *     charge).
 *   - Boundaries: n = 0 on the electrode planes (Sec. Methods, boundary
 *     conditions) realised as ghost cells k = -1 and k = nz that hold zero.
 *     Lateral faces are periodic or absorbing (zero ghosts) -- the paper only
 *     asks that Lx, Ly be large enough.
 *   - Tallies: the charge the update formula would place into an electrode
 *     ghost cell is the charge collected by that electrode during the step
 *     ("removed from the array as they reach either of the electrodes");
 *     the same for lateral ghosts when they absorb.  Recombined charge is
 *     alpha dt n+ n- summed over the cells.  f = collected / released
 *     (Eq. collection_efficiency).
 *
 * Grid reading: cell-centred, cell (i,j,k) spans [i dx, (i+1) dx) on each axis,
 * dx = dy = dz, gap d = nz dx.  Anode at z = 0, cathode at z = d; positive ions
 * drift to +z, negative ions to -z.
 *
 * All reductions are done per z-plane into an array and then summed in plane
 * order, so results do not depend on the OpenMP thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double dx, dt;
    double mu[2], D[2];   /* [0] = positive ions, [1] = negative ions */
    double alpha;         /* cm^3/s */
    double E;             /* V/cm, along +z */
    int lateral_bc;       /* 0 periodic, 1 absorbing */
    int scheme;           /* 0 blended (Lax-Wendroff) derivative, 1 pure upwind */
    double *n[2];         /* padded (nx+2)(ny+2)(nz+2), one ghost layer */
    double *nn[2];
    double *plane_work;   /* per-plane partial sums */
    double released[2], col_anode[2], col_cathode[2], lost_lateral[2];
    double recombined;
    int space_charge;     /* 1: include the -/+ mu n div E term */
    double sc_added[2];   /* ions added to each species by that term (negative: removed) */
    int64_t steps;
    double t;             /* simulated time: the sum of the steps' dt */
} orc_state;

/* Elementary charge (C) and vacuum permittivity (F/cm): div E = Q/EPS0 (n+ - n-)
 * with n in ions/cm^3 gives V/cm^2. */
static const double ORC_Q = 1.602176634e-19;
static const double ORC_EPS0 = 8.8541878128e-14;
/* sqrt(pi), the normalisation of the 1D profile exp(-u^2/b^2)/(sqrt(pi) b) */
static const double ORC_SQRT_PI = 1.7724538509055160272981674833411;

static inline size_t pidx(const orc_state *S, int i, int j, int k) {
    return ((size_t)(k + 1) * (size_t)(S->ny + 2) + (size_t)(j + 1)) * (size_t)(S->nx + 2) + (size_t)(i + 1);
}

orc_state *orc_create(int nx, int ny, int nz, double dx, double dt,
                      double mu_p, double mu_m, double D_p, double D_m,
                      double alpha, double E, int lateral_bc, int scheme) {
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dt > 0)) return NULL;
    orc_state *S = (orc_state *)calloc(1, sizeof(orc_state));
    if (!S) return NULL;
    S->nx = nx; S->ny = ny; S->nz = nz; S->dx = dx; S->dt = dt;
    S->mu[0] = mu_p; S->mu[1] = mu_m; S->D[0] = D_p; S->D[1] = D_m;
    S->alpha = alpha; S->E = E; S->lateral_bc = lateral_bc; S->scheme = scheme;
    size_t tot = (size_t)(nx + 2) * (ny + 2) * (nz + 2);
    for (int s = 0; s < 2; ++s) {
        S->n[s] = (double *)calloc(tot, sizeof(double));
        S->nn[s] = (double *)calloc(tot, sizeof(double));
        if (!S->n[s] || !S->nn[s]) return NULL;
    }
    S->plane_work = (double *)calloc((size_t)(nz + 2) * 16, sizeof(double));
    return S;
}

void orc_destroy(orc_state *S) {
    if (!S) return;
    for (int s = 0; s < 2; ++s) { free(S->n[s]); free(S->nn[s]); }
    free(S->plane_work);
    free(S);
}

/* Fraction of a 1D Gaussian of density exp(-u^2/b^2)/(sqrt(pi) b) that lies
 * in [lo, hi): half the difference of erf at the scaled edges. */
static double gauss_cell_weight(double lo, double hi, double centre, double b) {
    return 0.5 * (erf((hi - centre) / b) - erf((lo - centre) / b));
}

/* Deposit one batch of tracks parallel to z that span the gap.
 * x_cm, y_cm: track centres; let_keV_um: LET; b_cm: Gaussian radius; W_eV per
 * ion pair.  Eq. (linear_density): N0 = LET/W, with LET in keV/um converted to
 * eV/cm (x 1e7).  Each cell receives N0 * wx * wy / dx^2 (ions/cm^3) on every
 * z plane and for both species.  The window is +-ceil(6 b/dx) cells around the
 * cell that holds the centre.  Returns the released ions per species that
 * actually landed in the domain. */
double orc_deposit(orc_state *S, int64_t ntracks, const double *x_cm, const double *y_cm,
                   const double *let_keV_um, const double *b_cm, double W_eV) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const double dx = S->dx;
    double *plane = (double *)calloc((size_t)nx * ny, sizeof(double));
    for (int64_t t = 0; t < ntracks; ++t) {
        double N0 = let_keV_um[t] * 1e7 / W_eV;       /* ions per cm */
        double b = b_cm[t];
        int w = (int)ceil(6.0 * b / dx);
        int ic = (int)floor(x_cm[t] / dx), jc = (int)floor(y_cm[t] / dx);
        for (int jj = jc - w; jj <= jc + w; ++jj) {
            int j = jj;
            if (S->lateral_bc == 0) { j %= ny; if (j < 0) j += ny; }
            else if (j < 0 || j >= ny) continue;
            double wy = gauss_cell_weight(jj * dx, (jj + 1) * dx, y_cm[t], b);
            for (int ii = ic - w; ii <= ic + w; ++ii) {
                int i = ii;
                if (S->lateral_bc == 0) { i %= nx; if (i < 0) i += nx; }
                else if (i < 0 || i >= nx) continue;
                double wx = gauss_cell_weight(ii * dx, (ii + 1) * dx, x_cm[t], b);
                plane[(size_t)j * nx + i] += N0 * wx * wy / (dx * dx);
            }
        }
    }
    double sum = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) sum += plane[(size_t)j * nx + i];
    double released = sum * dx * dx * dx * nz;
    for (int s = 0; s < 2; ++s) {
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    S->n[s][pidx(S, i, j, k)] += plane[(size_t)j * nx + i];
        S->released[s] += released;
    }
    free(plane);
    return released;
}

/* Deposit tracks at an angle theta in [0, pi/2] to the field (Fig. setup (a)),
 * rotated in the x-z plane, each axis through (x_cm, y_cm, d/2).  Eq. (Gaussian)
 * about the axis: n = N0/(pi b^2) exp(-r^2/b^2), r the distance from the axis.
 * In the plane of cell centres z_k that distance has the components
 * u = (x - x0) cos(theta) - (z_k - d/2) sin(theta) and y - y0, so the plane holds
 * a Gaussian of width b/cos(theta) in x, centred where u = 0.  Each cell receives
 * its integral over the cell in x and y divided by the cell's area (the cell-
 * average reading), sampled at the cell centre in z:
 *   (N0/cos theta) wx wy / dx^2,  wx = (erf(u_hi/b) - erf(u_lo/b)) / 2,
 * over a window of +-ceil(6 b/(dx cos theta)) cells in x and +-ceil(6 b/dx) in
 * y.  Periodic faces wrap the window (the images of a tilted track are a
 * periodic array of parallel tracks, and their densities add), absorbing faces
 * clip it.  A track within cos(theta) dx/b < 1e-3 of parallel to the
 * electrodes is one track through the box instead: every cell once, with the
 * x integral taken at the cell centre, N0/(sqrt(pi) b) exp(-u_c^2/b^2) wy/dx
 * (the limit cos -> 0; at pi/2 the density does not depend on x).  theta = 0
 * gives orc_deposit's arithmetic.  Returns the released ions per species. */
double orc_deposit_angled(orc_state *S, int64_t ntracks, const double *x_cm, const double *y_cm,
                          const double *let_keV_um, const double *b_cm, const double *theta, double W_eV) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const double dx = S->dx, zmid = 0.5 * nz * dx;
    const size_t plane = (size_t)nx * ny;
    double *add = (double *)calloc(plane * nz, sizeof(double));
    for (int64_t t = 0; t < ntracks; ++t) {
        const double N0 = let_keV_um[t] * 1e7 / W_eV;   /* ions per cm */
        const double b = b_cm[t], c = cos(theta[t]), sn = sin(theta[t]);
        const int wy = (int)ceil(6.0 * b / dx);
        const int jc = (int)floor(y_cm[t] / dx);
        const int mid = c * dx / b < 1e-3;
        for (int k = 0; k < nz; ++k) {
            const double zk = (k + 0.5) * dx;
            for (int jj = jc - wy; jj <= jc + wy; ++jj) {
                int j = jj;
                if (S->lateral_bc == 0) { j %= ny; if (j < 0) j += ny; }
                else if (j < 0 || j >= ny) continue;
                const double wyv = gauss_cell_weight(jj * dx, (jj + 1) * dx, y_cm[t], b);
                double *row = add + (size_t)k * plane + (size_t)j * nx;
                if (mid) {
                    for (int i = 0; i < nx; ++i) {
                        const double u = ((i + 0.5) * dx - x_cm[t]) * c - (zk - zmid) * sn;
                        row[i] += N0 / (ORC_SQRT_PI * b) * exp(-(u * u) / (b * b)) * wyv / dx;
                    }
                    continue;
                }
                /* x where u = 0 in this plane, and the window about it */
                const double xc = x_cm[t] + (zk - zmid) * sn / c;
                const int wx = (int)ceil(6.0 * b / (dx * c));
                const int ic = (int)floor(xc / dx);
                for (int ii = ic - wx; ii <= ic + wx; ++ii) {
                    int i = ii;
                    if (S->lateral_bc == 0) { i %= nx; if (i < 0) i += nx; }
                    else if (i < 0 || i >= nx) continue;
                    const double wxv = gauss_cell_weight(ii * dx, (ii + 1) * dx, xc, b / c);
                    row[i] += (N0 / c) * wxv * wyv / (dx * dx);
                }
            }
        }
    }
    double sum = 0.0;
    for (size_t q = 0; q < plane * nz; ++q) sum += add[q];
    const double released = sum * dx * dx * dx;
    for (int s = 0; s < 2; ++s) {
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    S->n[s][pidx(S, i, j, k)] += add[(size_t)k * plane + (size_t)j * nx + i];
        S->released[s] += released;
    }
    free(add);
    return released;
}

/* Lateral ghost layers: copies of the opposite face when periodic, zero when
 * absorbing.  Electrode ghost planes always hold zero. */
static void fill_ghosts(orc_state *S, double *a) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    for (int k = -1; k <= nz; ++k) {
        for (int j = -1; j <= ny; ++j) {
            for (int i = -1; i <= nx; ++i) {
                int ghost_z = (k < 0 || k >= nz);
                int ghost_x = (i < 0 || i >= nx);
                int ghost_y = (j < 0 || j >= ny);
                if (!ghost_x && !ghost_y && !ghost_z) continue;
                double v = 0.0;
                if (!ghost_z && S->lateral_bc == 0) {
                    int ii = (i + nx) % nx, jj = (j + ny) % ny;
                    v = a[pidx(S, ii, jj, k)];
                }
                a[pidx(S, i, j, k)] = v;
            }
        }
    }
}

/* Value of the padded array, zero outside the padding. */
static inline double at(const orc_state *S, const double *a, int i, int j, int k) {
    if (i < -1 || i > S->nx || j < -1 || j > S->ny || k < -1 || k > S->nz) return 0.0;
    return a[pidx(S, i, j, k)];
}

/* The right-hand side of the discretised Eq. (theEquation) at one cell,
 * returned as the new value n^{l+1}.  sigma = +1 for n+, -1 for n-. */
static double update_cell(const orc_state *S, int s, int i, int j, int k, double rec, double divE) {
    const double *a = S->n[s];
    const double dx = S->dx, dt = S->dt;
    double n0 = at(S, a, i, j, k);
    double xp = at(S, a, i + 1, j, k), xm = at(S, a, i - 1, j, k);
    double yp = at(S, a, i, j + 1, k), ym = at(S, a, i, j - 1, k);
    double zp = at(S, a, i, j, k + 1), zm = at(S, a, i, j, k - 1);
    double dx2 = dx * dx;
    /* second derivatives, 3-point per axis */
    double lap = ((xp + xm) - 2.0 * n0) / dx2 + ((yp + ym) - 2.0 * n0) / dx2
               + ((zp + zm) - 2.0 * n0) / dx2;
    /* drift velocity along z: +mu E for positive ions, -mu E for negative */
    double sigma = (s == 0) ? 1.0 : -1.0;
    double v = sigma * S->mu[s] * S->E;
    double c = fabs(v) * dt / dx;
    double central = (zp - zm) / (2.0 * dx);
    double upwind = (v >= 0.0) ? (n0 - zm) / dx : (zp - n0) / dx;
    double dndz = (S->scheme == 0) ? c * upwind + (1.0 - c) * central : upwind;
    /* space charge: -/+ mu n div E (zero unless enabled) */
    double sc = sigma * S->mu[s] * n0 * divE;
    return n0 + dt * (S->D[s] * lap - v * dndz - rec - sc);
}

/* One explicit time step of both species with tallies. */
void orc_step(orc_state *S) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const double vol = S->dx * S->dx * S->dx;
    for (int s = 0; s < 2; ++s) fill_ghosts(S, S->n[s]);
    const int absorbing = (S->lateral_bc == 1);
    double *W = S->plane_work;            /* 16 partials per plane index k+1 */
    memset(W, 0, sizeof(double) * (size_t)(nz + 2) * 16);
#pragma omp parallel for schedule(static)
    for (int k = -1; k <= nz; ++k) {
        double *w = W + (size_t)(k + 1) * 16;
        int ghost_z = (k < 0 || k >= nz);
        for (int j = -1; j <= ny; ++j) {
            for (int i = -1; i <= nx; ++i) {
                int gx = (i < 0 || i >= nx), gy = (j < 0 || j >= ny);
                int nghost = gx + gy + ghost_z;
                if (nghost == 0) {
                    double np = S->n[0][pidx(S, i, j, k)], nm = S->n[1][pidx(S, i, j, k)];
                    double rec = S->alpha * (np * nm);   /* symmetric in n+, n- */
                    double divE = S->space_charge ? (ORC_Q / ORC_EPS0) * (np - nm) : 0.0;
                    for (int s = 0; s < 2; ++s)
                        S->nn[s][pidx(S, i, j, k)] = update_cell(S, s, i, j, k, rec, divE);
                    w[0] += S->alpha * S->dt * np * nm * vol;
                    if (S->space_charge) {
                        w[7] -= S->dt * S->mu[0] * np * divE * vol;   /* n+: -mu+ n+ div E */
                        w[8] += S->dt * S->mu[1] * nm * divE * vol;   /* n-: +mu- n- div E */
                    }
                } else if (nghost == 1) {
                    /* a ghost cell next to the domain: what the update would
                     * move into it leaves the domain through that face */
                    if (!ghost_z && !absorbing) continue;   /* periodic copy */
                    for (int s = 0; s < 2; ++s) {
                        double out = update_cell(S, s, i, j, k, 0.0, 0.0) * vol;
                        if (ghost_z) w[(k < 0 ? 1 : 3) + s] += out;   /* 1,2 anode; 3,4 cathode */
                        else w[5 + s] += out;                         /* lateral */
                    }
                }
            }
        }
    }
    double rec = 0, ca[2] = {0, 0}, cc[2] = {0, 0}, ll[2] = {0, 0}, sa[2] = {0, 0};
    for (int k = 0; k < nz + 2; ++k) {
        double *w = W + (size_t)k * 16;
        rec += w[0];
        for (int s = 0; s < 2; ++s) { ca[s] += w[1 + s]; cc[s] += w[3 + s]; ll[s] += w[5 + s]; sa[s] += w[7 + s]; }
    }
    S->recombined += rec;
    for (int s = 0; s < 2; ++s) {
        S->col_anode[s] += ca[s]; S->col_cathode[s] += cc[s]; S->lost_lateral[s] += ll[s];
        S->sc_added[s] += sa[s];
        double *t = S->n[s]; S->n[s] = S->nn[s]; S->nn[s] = t;
    }
    S->steps += 1;
    S->t += S->dt;
}

/* Change the time step for the steps that follow (the step-size ladder of a
 * run to completion).  Returns 0, or -1 for a dt that is not positive. */
int orc_set_dt(orc_state *S, double dt) {
    if (!(dt > 0)) return -1;
    S->dt = dt;
    return 0;
}

/* Simulated time so far: the sum of the dt of every step taken. */
double orc_time(const orc_state *S) { return S->t; }

void orc_steps(orc_state *S, int64_t n) { for (int64_t l = 0; l < n; ++l) orc_step(S); }

/* Ions of each species still in the domain, and the extreme densities. */
void orc_in_domain(const orc_state *S, double *out2, double *minmax4) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const double vol = S->dx * S->dx * S->dx;
    for (int s = 0; s < 2; ++s) {
        double sum = 0, mn = INFINITY, mx = -INFINITY;
        for (int k = 0; k < nz; ++k) {
            double ps = 0;
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double v = S->n[s][pidx(S, i, j, k)];
                    ps += v;
                    if (v < mn) mn = v;
                    if (v > mx) mx = v;
                }
            sum += ps;
        }
        out2[s] = sum * vol;
        if (minmax4) { minmax4[2 * s] = mn; minmax4[2 * s + 1] = mx; }
    }
}

/* tallies: released[2], col_anode[2], col_cathode[2], lost_lateral[2], recombined, steps */
void orc_tallies(const orc_state *S, double *out10) {
    for (int s = 0; s < 2; ++s) {
        out10[0 + s] = S->released[s];
        out10[2 + s] = S->col_anode[s];
        out10[4 + s] = S->col_cathode[s];
        out10[6 + s] = S->lost_lateral[s];
    }
    out10[8] = S->recombined;
    out10[9] = (double)S->steps;
}

/* Space-charge term on (1) or off (0). */
void orc_set_space_charge(orc_state *S, int on) { S->space_charge = on ? 1 : 0; }

/* Ions added to each species by the space-charge term so far (negative: removed). */
void orc_space_charge(const orc_state *S, double *out2) {
    out2[0] = S->sc_added[0];
    out2[1] = S->sc_added[1];
}

/* Copy one species' interior densities to dst laid out [nz][ny][nx]. */
void orc_get_density(const orc_state *S, int s, double *dst) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                dst[((size_t)k * ny + j) * nx + i] = S->n[s][pidx(S, i, j, k)];
}

/* Set both species' interior densities ([nz][ny][nx], ions/cm^3) as an initial
 * condition: all tallies restart and the released charge is what was set. */
void orc_set_density(orc_state *S, const double *plus, const double *minus) {
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const double vol = S->dx * S->dx * S->dx;
    const double *src[2] = {plus, minus};
    for (int s = 0; s < 2; ++s) {
        memset(S->n[s], 0, sizeof(double) * (size_t)(nx + 2) * (ny + 2) * (nz + 2));
        double sum = 0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double v = src[s][((size_t)k * ny + j) * nx + i];
                    S->n[s][pidx(S, i, j, k)] = v;
                    sum += v;
                }
        S->released[s] = sum * vol;
        S->col_anode[s] = S->col_cathode[s] = S->lost_lateral[s] = 0;
        S->sc_added[s] = 0;
    }
    S->recombined = 0;
    S->steps = 0;
}
