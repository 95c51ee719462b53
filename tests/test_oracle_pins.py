"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an exact discrete invariant of the scheme, a published value, or a library
routine that computes the same special function another way.  A dropped term,
a wrong sign or index, or a transposed operand in the oracle fails at least
one of them (see the comment on each test).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

import oracle.oracle as o
from paper_1610_06749_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MU, DD, ALPHA = (1.73, 1.87), (0.037, 0.037), 1.6e-6


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# seeded inputs
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    g = _gold("splitmix64.json")["vectors"]
    got0 = [format(int(v), "016x") for v in synth.splitmix64(g[0]["seed"], 3)]
    assert got0 == g[0]["outputs_hex"]
    got1 = [str(int(v)) for v in synth.splitmix64(g[1]["seed"], 3)]
    assert got1 == g[1]["outputs_dec"]


def test_uniform_tracks_are_reproducible_and_in_range():
    a = synth.uniform_tracks(42, 500, 0.1, 0.2, 1e-3)
    b = synth.uniform_tracks(42, 500, 0.1, 0.2, 1e-3)
    assert np.array_equal(a.x_cm, b.x_cm) and np.array_equal(a.let_keV_um, b.let_keV_um)
    assert a.x_cm.min() >= 0 and a.x_cm.max() < 0.1 and a.y_cm.max() < 0.2
    assert a.let_keV_um.min() >= 1.0 and a.let_keV_um.max() < 1000.0


def test_poisson_arrival_count_matches_rate():
    # mean count lambda*T with lambda = rate*Lx*Ly; 5 sigma band
    rate, L, dt, n = 1e7, 0.05, 1e-8, 20000
    tr = synth.poisson_tracks(7, rate, L, L, dt, n, 1e-3, synth.CONTINUOUS_LET)
    lam_T = rate * L * L * dt * n
    assert abs(len(tr) - lam_T) < 5 * math.sqrt(lam_T)
    assert np.all(np.diff(tr.step) >= 0) and tr.step.max() < n
    frac20 = np.mean(tr.let_keV_um == 20.0)
    assert abs(frac20 - 0.7) < 5 * math.sqrt(0.21 / len(tr))


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.1, 1.0, 5.0, 20.0, 39.9, 40.1, 80.0, 300.0])
def test_ei_matches_scipy_expi(x):
    # own series / asymptotic code vs an independent library implementation
    ref = sp.expi(x) * math.exp(-x)
    assert o.ei_scaled(x) == pytest.approx(ref, rel=2e-13, abs=1e-15)


@pytest.mark.parametrize("let", [1e-3, 0.03, 0.115, 1.02, 10.0, 100.0, 1000.0])
def test_jaffe_printed_form_equals_integral_form(let):
    # Eq. (Jaffe_noangle) through Ei vs its integral representation
    E = 2000.0
    a = o.jaffe_parallel(let, 1e-3, 0.2, E, 1.73, 0.0356, ALPHA, method="ei")
    b = o.jaffe_parallel(let, 1e-3, 0.2, E, 1.73, 0.0356, ALPHA, method="quad")
    assert a == pytest.approx(b, rel=1e-10)
    assert 0.0 < a <= 1.0


def test_jaffe_limits():
    # y1 -> infinity (no recombination): f -> 1; the integral is bounded by
    # its end-point values: 1/(1 + ln(1+y2)/y1) <= f <= 1
    f = o.jaffe_parallel(1e-6, 1e-3, 0.02, 1e4, 1.8, 0.037, ALPHA)
    assert f == pytest.approx(1.0, abs=1e-6)
    y1, y2 = o.jaffe_y(10.0, 1e-3, 0.02, 1e4, 1.8, 0.037, ALPHA)
    f = o.jaffe_parallel(10.0, 1e-3, 0.02, 1e4, 1.8, 0.037, ALPHA)
    assert 1.0 / (1.0 + math.log1p(y2) / y1) <= f <= 1.0


def test_jaffe_config1_value_and_paper_table_ions():
    # y1 = 8 pi D/(alpha N0), y2 = 2 d D/(mu b^2 E) for 100 keV/um, b = 10 um,
    # d = 200 um, 200 V, mean mu 1.80, D 0.037
    y1, y2 = o.jaffe_y(100.0, 1e-3, 0.02, 1e4, 1.80, 0.037, ALPHA)
    N0 = 100.0 * 1e7 / 34.0
    assert y1 == pytest.approx(8 * math.pi * 0.037 / (ALPHA * N0), rel=1e-14)
    assert y1 == pytest.approx(0.019761, rel=1e-4) and y2 == pytest.approx(0.082222, rel=1e-4)
    assert o.jaffe_parallel(100.0, 1e-3, 0.02, 1e4, 1.80, 0.037, ALPHA) == pytest.approx(0.39835, abs=5e-6)


def test_jaffe_angle_uses_modified_bessel_identity():
    # (i pi/2) H0^(1)(iZ) = K0(Z) for real Z > 0 (Eq. angle)
    for Z in [0.1, 1.0, 7.5]:
        h = (1j * math.pi / 2) * sp.hankel1(0, 1j * Z)
        assert h.real == pytest.approx(sp.k0(Z), rel=1e-12) and abs(h.imag) < 1e-12
    # theta = 0 gives Z = 0 and S -> infinity, so f -> 0 is not the parallel
    # limit (the formula holds at large angles only); at theta = pi/2 it is
    # bounded by 1
    f = o.jaffe_angle(0.115, 2e-3, 2000.0, math.pi / 2, 1.73, 0.0356, ALPHA)
    assert 0 < f < 1


@pytest.mark.parametrize("u,f", [(0.5, 0.81093), (1.0, 0.69315), (2.0, 0.54931), (5.0, 0.35835)])
def test_boag_2vm_values(u, f):
    assert o.boag_2vm(u) == pytest.approx(f, abs=5e-6)


def test_dt_rule_sits_on_the_von_neumann_bound():
    # Eq. (vNeum): 2(sx+sy+sz) + cz^2 = 1 for the limiting species at dt_vN
    dx, V, d = 2e-4, 200.0, 0.02
    dt = o.dt_von_neumann(dx, V, d, MU, DD)
    E = V / d
    vals = [6 * D * dt / dx ** 2 + (m * E * dt / dx) ** 2 for m, D in zip(MU, DD)]
    assert max(vals) == pytest.approx(1.0, rel=1e-12)
    assert all(v <= 1.0 + 1e-12 for v in vals)
    dtu = o.dt_von_neumann(dx, V, d, MU, DD, scheme=o.SCHEME_UPWIND)
    vals = [6 * D * dtu / dx ** 2 + (m * E * dtu / dx) for m, D in zip(MU, DD)]
    assert max(vals) == pytest.approx(1.0, rel=1e-12)
    # reaction bound alpha dt n_peak = kappa
    npk = o.peak_track_density([1000.0], [1e-3])
    assert npk == pytest.approx(1000.0 * 1e7 / 34.0 / (math.pi * 1e-6), rel=1e-14)
    dtr = o.dt_rule(5e-4, 50.0, 0.2, MU, DD, ALPHA, n_peak=npk, kappa=0.5)
    assert ALPHA * dtr * npk == pytest.approx(0.5, rel=1e-14)


# --------------------------------------------------------------------------
# deposition (Eqs. linear_density, Gaussian, created, unity)
# --------------------------------------------------------------------------

def test_deposit_periodic_releases_N0_times_gap():
    # Eq. (created): N_released = N0 * l exactly when nothing is clipped
    O = o.Oracle(24, 20, 7, 5e-4, 1e-9, lateral_bc=o.LATERAL_PERIODIC)
    tr = synth.uniform_tracks(3, 11, 24 * 5e-4, 20 * 5e-4, 1e-3)
    rel = O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
    want = float(np.sum(tr.let_keV_um * 1e7 / 34.0)) * 7 * 5e-4
    assert rel == pytest.approx(want, rel=1e-12)
    t = O.tallies()
    assert t.in_domain[0] == pytest.approx(want, rel=1e-12)
    assert np.array_equal(O.density(0), O.density(1))
    # z-independent: every plane is identical
    n = O.density(0)
    assert np.array_equal(n[0], n[6])


def test_deposit_absorbing_clips_the_gaussian_tail():
    # a track a distance a from one face loses erfc(a/b)/2 of its charge
    # (a 1D Gaussian of density exp(-x^2/b^2)/(sqrt(pi) b)): b is not sigma
    dx, b = 2e-4, 1e-3
    nx = 60
    a = 3.3e-4
    O = o.Oracle(nx, nx, 3, dx, 1e-9, lateral_bc=o.LATERAL_ABSORBING)
    rel = O.deposit([a], [nx * dx / 2], [1.0], [b])
    full = 1.0 * 1e7 / 34.0 * 3 * dx
    want = full * (1.0 - 0.5 * math.erfc(a / b))
    assert rel == pytest.approx(want, rel=1e-10)


def test_deposit_cell_density_matches_point_gaussian_at_fine_grid():
    # Eq. (Gaussian) n0(r) = N0/(pi b^2) exp(-r^2/b^2) sampled at cell centres,
    # and Eq. (unity): Simpson's rule over the plane gives I0 = N0.
    b, dx, nx = 1e-3, 5e-5, 200        # dx = b/20, Lx = 10 b (Fig. 2 grid rule)
    O = o.Oracle(nx, nx, 1, dx, 1e-12, lateral_bc=o.LATERAL_ABSORBING)
    xc = yc = nx * dx / 2 + 0.3 * dx
    O.deposit([xc], [yc], [0.115], [b])
    plane = O.density(0)[0]
    N0 = 0.115 * 1e7 / 34.0
    xs = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(xs, xs)
    point = N0 / (math.pi * b * b) * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / b ** 2)
    assert np.max(np.abs(plane - point)) / point.max() < 2e-3
    I0 = integrate.simpson(integrate.simpson(point, x=xs, axis=1), x=xs)
    assert I0 / N0 == pytest.approx(1.0, abs=1e-6)
    # cell averages conserve exactly the mass inside the box: the product of
    # the 1D Gaussian masses between the faces (a tail of ~erfc(5) is outside)
    L = nx * dx
    inside = (0.5 * (math.erf((L - xc) / b) + math.erf(xc / b))) ** 2
    assert plane.sum() * dx * dx / N0 == pytest.approx(inside, rel=1e-13)
    assert 1.0 - inside > 1e-12


# --------------------------------------------------------------------------
# transport invariants (Appendix scheme)
# --------------------------------------------------------------------------

def _plane_variance(m, dx):
    ny, nx = m.shape
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    w = m / m.sum()
    mx = np.sum(w * x[None, :]); my = np.sum(w * y[:, None])
    vx = np.sum(w * (x[None, :] - mx) ** 2); vy = np.sum(w * (y[:, None] - my) ** 2)
    return vx, vy


def test_pure_diffusion_variance_grows_2Ddt_per_step_and_follows_closed_form():
    # FTCS is a lattice random walk: on a plane whose z-neighbours hold the
    # same values (the mid-plane of a z-uniform track, before the electrodes
    # are felt there: one cell per step) each lateral variance grows by
    # exactly 2 D dt per step; the profile follows Eq. (Gaussian) with
    # b^2 -> b^2 + 4 D t.
    b, dx, nx, nz = 1e-3, 2e-4, 60, 90
    D = (0.037, 0.05)
    dt = 2e-9
    steps = 40
    O = o.Oracle(nx, nx, nz, dx, dt, mu=(0, 0), D=D, alpha=0.0, voltage_V=0.0,
                 lateral_bc=o.LATERAL_PERIODIC)
    c = nx * dx / 2
    O.deposit([c], [c], [1.0], [b])
    v0 = [_plane_variance(O.density(s)[nz // 2], dx) for s in range(2)]
    O.step(steps)
    for s in range(2):
        vx, vy = _plane_variance(O.density(s)[nz // 2], dx)
        inc = 2 * D[s] * dt * steps
        assert vx - v0[s][0] == pytest.approx(inc, rel=1e-9)
        assert vy - v0[s][1] == pytest.approx(inc, rel=1e-9)
    # shape against the closed form (mid-plane, normalised)
    n = O.density(0)[nz // 2]
    xs = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(xs, xs)
    ref = o.gaussian_track_diffused(np.hypot(X - c, Y - c), dt * steps, 1.0, b, D[0])
    err = np.max(np.abs(n / n.sum() - ref / ref.sum())) / np.max(ref / ref.sum())
    assert err < 1e-2


@pytest.mark.parametrize("m", [1, 3])
def test_z_sine_mode_is_an_eigenvector_with_dirichlet_electrodes(m):
    # n_k = sin(pi m (k+1)/(nz+1)) with n = 0 at k = -1 and k = nz decays by
    # 1 - 4 s_z sin^2(pi m / (2(nz+1))) per step (3-point Laplacian)
    nz, dx, dt, D = 30, 1e-3, 5e-9, 0.04
    O = o.Oracle(4, 4, nz, dx, dt, mu=(0, 0), D=(D, D), alpha=0.0, voltage_V=0.0)
    k = np.arange(nz)
    prof = np.sin(math.pi * m * (k + 1) / (nz + 1))
    field = np.broadcast_to(prof[:, None, None], (nz, 4, 4)) * 1e9
    O.set_density(field, field)
    steps = 25
    O.step(steps)
    s = D * dt / dx ** 2
    lam = 1.0 - 4.0 * s * math.sin(math.pi * m / (2 * (nz + 1))) ** 2
    got = O.density(0)[:, 1, 2]
    np.testing.assert_allclose(got, prof * 1e9 * lam ** steps, rtol=1e-12, atol=1e-12 * 1e9)
    t = O.tallies()
    assert t.released[0] == pytest.approx(t.in_domain[0] + t.collected[0], rel=1e-13)


def _z_blob(nz, k0, w):
    k = np.arange(nz)
    return np.exp(-((k - k0) / w) ** 2)


@pytest.mark.parametrize("scheme", [o.SCHEME_LAX_WENDROFF, o.SCHEME_UPWIND])
def test_drift_moments(scheme):
    # Lax-Wendroff: centroid moves c dx per step, variance grows 2 s_z dx^2.
    # Upwind: centroid c dx, variance 2 s_z dx^2 + c (1 - c) dx^2.
    # Positive ions move to +z, negative ions to -z.
    nz, dx, V = 200, 1e-3, 40.0
    D = (0.02, 0.03)
    mu = (1.36, 2.10)
    dt = 0.5 * o.dt_von_neumann(dx, V, nz * dx, mu, D, scheme)
    O = o.Oracle(2, 2, nz, dx, dt, mu=mu, D=D, alpha=0.0, voltage_V=V, scheme=scheme)
    blob = _z_blob(nz, 100.0, 6.0)
    f = np.broadcast_to(blob[:, None, None], (nz, 2, 2))
    O.set_density(f, f)
    def moments(s):
        p = O.density(s)[:, 0, 0]
        k = np.arange(nz)
        w = p / p.sum()
        m = np.sum(w * k)
        return m, np.sum(w * (k - m) ** 2)
    m0 = [moments(s) for s in range(2)]
    steps = 30
    O.step(steps)
    E = V / (nz * dx)
    for s, sign in ((0, 1.0), (1, -1.0)):
        c = mu[s] * E * dt / dx
        sz = D[s] * dt / dx ** 2
        m1, v1 = moments(s)
        assert m1 - m0[s][0] == pytest.approx(sign * c * steps, rel=1e-9)
        dv = 2 * sz + (c * (1 - c) if scheme == o.SCHEME_UPWIND else 0.0)
        assert v1 - m0[s][1] == pytest.approx(dv * steps, rel=1e-8)


def test_lax_wendroff_at_c_equal_one_is_an_exact_shift():
    # c = 1, s = 0: every carrier moves exactly one cell per step.  All
    # quantities are powers of two so that c is exactly 1.
    nz = 16
    dx = 2.0 ** -10
    O = o.Oracle(1, 1, nz, dx, dx, mu=(1.0, 1.0), D=(0.0, 0.0), alpha=0.0,
                 voltage_V=nz * dx)
    p = np.zeros((nz, 1, 1)); p[3, 0, 0] = 5.0; p[4, 0, 0] = 7.0
    O.set_density(p, p)
    O.step(2)
    a = O.density(0)[:, 0, 0]; bneg = O.density(1)[:, 0, 0]
    want_p = np.zeros(nz); want_p[5] = 5.0; want_p[6] = 7.0
    want_m = np.zeros(nz); want_m[1] = 5.0; want_m[2] = 7.0
    assert np.array_equal(a, want_p) and np.array_equal(bneg, want_m)
    O.step(1)       # n- now at cells 0, 1 (5 and 7): nothing has reached the anode
    t = O.tallies()
    assert t.collected_anode[1] == 0.0
    O.step(1)
    t = O.tallies()
    assert t.collected_anode[1] == 5.0 * dx ** 3
    O.step(1)
    t = O.tallies()
    assert t.collected_anode[1] == 12.0 * dx ** 3 and t.collected_cathode[1] == 0.0
    assert t.in_domain[1] == 0.0


@pytest.mark.parametrize("bc", [o.LATERAL_PERIODIC, o.LATERAL_ABSORBING])
def test_charge_conservation_with_and_without_recombination(bc):
    # released = in domain + collected + lost laterally + recombined, every
    # step; the collected charge comes from the electrode ghost cells, not
    # from the sums, so this is not an identity of the bookkeeping.
    nx, nz, dx = 20, 30, 5e-4
    for alpha in (0.0, ALPHA):
        tr = synth.uniform_tracks(11, 9, nx * dx, nx * dx, 1.5e-3, let=("mixture", [(50.0, 1.0)]))
        dt = o.dt_rule(dx, 100.0, nz * dx, MU, DD, alpha, n_peak=o.peak_track_density(tr.let_keV_um, tr.b_cm))
        O = o.Oracle(nx, nx, nz, dx, dt, alpha=alpha, voltage_V=100.0, lateral_bc=bc)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        for _ in range(6):
            O.step(7)
            t = O.tallies()
            for s in range(2):
                total = t.in_domain[s] + t.collected[s] + t.lost_lateral[s] + t.recombined
                assert total == pytest.approx(t.released[s], rel=1e-12)
        if alpha == 0.0:
            assert t.recombined == 0.0
        if bc == o.LATERAL_PERIODIC:
            assert np.all(t.lost_lateral == 0.0)


def test_recombination_recurrence_and_continuum_limit():
    # E = 0, D = 0, uniform n+ = n- = n0: n <- n - alpha dt n^2 exactly, and
    # n(t) -> n0/(1 + alpha n0 t) as dt -> 0 with error O(alpha n0 dt)
    n0, T = 4e12, 2e-6
    errs = []
    for nsteps in (50, 100, 200):
        dt = T / nsteps
        O = o.Oracle(3, 3, 4, 1e-3, dt, mu=(0, 0), D=(0, 0), alpha=ALPHA, voltage_V=0.0)
        f = np.full((4, 3, 3), n0)
        O.set_density(f, f)
        O.step(nsteps)
        n = n0
        for _ in range(nsteps):
            n = n - ALPHA * dt * n * n
        got = O.density(0)
        assert np.all(got == got[0, 0, 0]) and np.array_equal(got, O.density(1))
        assert got[0, 0, 0] == pytest.approx(n, rel=1e-14)
        errs.append(abs(got[0, 0, 0] - n0 / (1 + ALPHA * n0 * T)))
    assert errs[1] < 0.55 * errs[0] and errs[2] < 0.55 * errs[1]   # first order in dt


def test_mirror_symmetry_is_bitwise():
    # mu+ = mu-, D+ = D-: n+(i,j,k) = n-(i,j,nz-1-k) at every step; anode and
    # cathode collections swap.  Catches a wrong upwind side or drift sign.
    nx, nz, dx = 16, 24, 5e-4
    tr = synth.uniform_tracks(5, 6, nx * dx, nx * dx, 1e-3)
    dt = o.dt_rule(dx, 150.0, nz * dx, (1.8, 1.8), (0.04, 0.04), ALPHA,
                   n_peak=o.peak_track_density(tr.let_keV_um, tr.b_cm))
    O = o.Oracle(nx, nx, nz, dx, dt, mu=(1.8, 1.8), D=(0.04, 0.04), alpha=ALPHA,
                 voltage_V=150.0, lateral_bc=o.LATERAL_ABSORBING)
    O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
    for _ in range(4):
        O.step(5)
        assert np.array_equal(O.density(0), O.density(1)[::-1])
    t = O.tallies()
    assert t.collected_anode[0] == t.collected_cathode[1]
    assert t.collected_cathode[0] == t.collected_anode[1]


# --------------------------------------------------------------------------
# physics pins: Jaffe (initial recombination) and Boag (general recombination)
# --------------------------------------------------------------------------

def _single_track_f(let, b=1e-3, dx=2e-4, V=200.0, gap=0.02, mu=MU, D=DD, tol=1e-9):
    nz = int(round(gap / dx)); nxy = int(round(9.6 * b / dx))
    dt = o.dt_rule(dx, V, gap, mu, D, ALPHA, n_peak=o.peak_track_density([let], [b]))
    O = o.Oracle(nxy, nxy, nz, dx, dt, mu=mu, D=D, alpha=ALPHA, voltage_V=V,
                 lateral_bc=o.LATERAL_ABSORBING)
    c = 0.5 * nxy * dx
    O.deposit([c], [c], [let], [b])
    for _ in range(400):
        O.step(25)
        t = O.tallies()
        if t.in_domain.sum() / t.released.sum() < tol:
            break
    return t


@pytest.mark.parametrize("let,tol", [(0.1, 1e-4), (1.0, 5e-4), (3.0, 2e-3)])
def test_single_track_matches_jaffe_where_its_gaussian_ansatz_holds(let, tol):
    # Eq. (Jaffe_noangle) with mean mu and D (reading of the text beside it)
    # for a track parallel to E; 48x48x100 cells at dx = b/5, 200 V over 200 um.
    t = _single_track_f(let)
    fj = o.jaffe_parallel(let, 1e-3, 0.02, 1e4, 0.5 * sum(MU), 0.5 * sum(DD), ALPHA)
    assert abs(t.f - fj) < tol


@pytest.mark.slow
def test_single_track_jaffe_gap_shrinks_with_dx():
    # Sec. Stability and accuracy (ii): f converges as dx decreases
    fj = o.jaffe_parallel(1.0, 1e-3, 0.02, 1e4, 1.80, 0.037, ALPHA)
    e5 = abs(_single_track_f(1.0, dx=2e-4).f - fj)
    e10 = abs(_single_track_f(1.0, dx=1e-4).f - fj)
    assert e10 < 0.3 * e5 and e10 < 5e-5


def test_config1_jaffe_gap_is_a_converged_gap_not_discretisation():
    # The 100 keV/um single track (y1 = 0.02).  tests/golden/single_track_dx_sweep.json
    # holds the oracle's f at dx = b/5, b/10 and b/20 (written by the script
    # beside it); the b/5 value is rerun here.  The successive changes of f
    # shrink (the scheme converges; about first order, since the step is
    # drift-limited, dt ~ dx, and the explicit recombination is first order
    # in dt), while the gap to Eq. (Jaffe_noangle) grows towards ~0.058: the
    # gap is the Gaussian-shape ansatz behind Jaffe's form failing at this
    # LET, not discretisation error.
    g = _gold("single_track_dx_sweep.json")
    r5 = g["runs"][0]
    dt = o.dt_rule(r5["dx_cm"], g["voltage_V"], g["gap_cm"], n_peak=o.peak_track_density([g["LET_keV_um"]],
                                                                                        [g["b_cm"]]))
    assert dt == r5["dt_s"]
    O = o.Oracle(r5["nx"], r5["ny"], r5["nz"], r5["dx_cm"], dt, voltage_V=g["voltage_V"],
                 lateral_bc=o.LATERAL_ABSORBING)
    c = 0.5 * r5["nx"] * r5["dx_cm"]
    O.deposit([c], [c], [g["LET_keV_um"]], [g["b_cm"]])
    steps, done, _ = O.run_to_completion(tol=1e-9, check_every=32)
    assert done and steps == r5["steps"]
    assert O.tallies().f == pytest.approx(r5["f"], abs=1e-12)
    fj = o.jaffe_parallel(g["LET_keV_um"], g["b_cm"], g["gap_cm"], g["voltage_V"] / g["gap_cm"],
                          0.5 * sum(MU), 0.5 * sum(DD), ALPHA)
    assert fj == pytest.approx(g["f_jaffe"], abs=1e-14)
    f = [r["f"] for r in g["runs"]]
    d1, d2 = f[1] - f[0], f[2] - f[1]
    assert 0.0 < d2 < 0.7 * d1
    r = d2 / d1
    f_inf = f[2] + d2 * r / (1.0 - r)          # geometric (Richardson) extrapolation
    assert 0.05 < f_inf - fj < 0.07
    assert f[0] - fj < f[1] - fj < f[2] - fj


def test_proton_initial_recombination_below_0p1_percent():
    # Table 1 proton (LET 7.76e-4 keV/um, b = 10 um): 1 - f < 1e-3
    g = _gold("paper_tables.json")
    p = g["table1_track_parameters"]["proton"]
    t = _single_track_f(p["LET_keV_um"], b=p["b_um"] * 1e-4)
    assert 0.0 <= 1.0 - t.f < g["proton_initial_recombination_bound"]["one_minus_f_max"]


@pytest.mark.parametrize("u", [0.5, 1.0, 2.0, 5.0])
def test_uniform_slab_follows_boag_two_voltage_method(u):
    # A laterally uniform slab n over the whole gap released by one pulse:
    # f = ln(1+u)/u, u = alpha/(mu+ + mu-) n d^2 / V.  The diffusion
    # broadening of the fronts is the expected residual.
    nz, dx, V = 400, 5e-4, 200.0
    d = nz * dx
    n = u * (MU[0] + MU[1]) * V / (ALPHA * d * d)
    dt = o.dt_rule(dx, V, d, MU, DD, ALPHA, n_peak=n)
    O = o.Oracle(4, 4, nz, dx, dt, alpha=ALPHA, voltage_V=V)
    f = np.full((nz, 4, 4), n)
    O.set_density(f, f)
    while True:
        O.step(200)
        t = O.tallies()
        if t.in_domain.sum() / t.released.sum() < 1e-9:
            break
    assert t.f == pytest.approx(o.boag_2vm(u), abs=1e-2)


def _run_to_completion(O, tol=1e-6, chunk=100, cap=200000):
    while True:
        O.step(chunk)
        t = O.tallies()
        if t.in_domain.sum() / t.released.sum() < tol or t.steps >= cap:
            return t


def test_f_converges_at_first_order_in_the_reaction_bound():
    # The reaction-stability reading dt = min(dt_vN, kappa / (alpha n_peak)).
    # Explicit recombination is first order in dt, so with the bound active
    # successive halvings of kappa change f by half as much each time; from
    # kappa = 0.25 a halving moves f by less than 1e-3.  On this dense field
    # (LET up to 1000 keV/um) kappa = 0.5 moves f by about 2e-3, an error of
    # about 4e-3 against dt -> 0.  A second-order or missing reaction term, or
    # a bound that is not active, breaks the ratio.
    nx, ny, nz, dx, V = 24, 24, 40, 5e-4, 200.0
    tr = synth.uniform_tracks(9, 12, nx * dx, ny * dx, 1e-3, let="loguniform")
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
    fs = []
    for kappa in (0.5, 0.25, 0.125):
        dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, kappa=kappa, scheme=o.SCHEME_UPWIND)
        assert dt < o.dt_von_neumann(dx, V, nz * dx, MU, DD, scheme=o.SCHEME_UPWIND)   # the bound is active
        O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V, scheme=o.SCHEME_UPWIND)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        fs.append(_run_to_completion(O).f)
    d1, d2 = fs[1] - fs[0], fs[2] - fs[1]
    assert 0.0 < fs[0] < 1.0 and d1 > 0 and d2 > 0
    assert 1.7 < d1 / d2 < 2.5
    assert d2 < 1e-3 < d1


def test_many_overlapping_low_let_tracks_follow_boag():
    # Many proton-like tracks (LET ~4e-3 keV/um, spaced at b) released at
    # once: initial recombination is negligible, the tracks merge into a
    # nearly uniform charge density n = released / (Lx Ly d), and f follows
    # Boag's pulsed-beam f = ln(1+u)/u with u = alpha n d^2 / ((mu+ + mu-) V)
    # (the 2VM formula of Sec. "The free-electron component" at p = 0, used
    # again in Sec. "Comparison with Boag's free-electron models").  Track structure and the diffusion of the fronts are
    # the residual.
    nx, ny, nz, dx, V, b = 24, 24, 40, 5e-4, 200.0, 1e-3
    d = nz * dx
    g = (np.arange(12) + 0.5) * (nx * dx / 12)
    xs, ys = [a.ravel() for a in np.meshgrid(g, g)]
    u_target = 1.0
    n = u_target * (MU[0] + MU[1]) * V / (ALPHA * d * d)
    let = n * 34.0 * (nx * dx) * (ny * dx) / (xs.size * 1e7)
    dt = o.dt_rule(dx, V, d, MU, DD, ALPHA, n_peak=o.peak_track_density([let], [b]))
    O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V)
    O.deposit(xs, ys, np.full(xs.size, let), np.full(xs.size, b))
    t = _run_to_completion(O)
    n_rel = t.released[0] / ((nx * dx) * (ny * dx) * d)
    u = o.boag_u(ALPHA, MU[0], MU[1], n_rel, d, V)
    assert u == pytest.approx(u_target, rel=1e-6)
    assert t.f == pytest.approx(o.boag_2vm(u), abs=2e-2)


def test_upwind_stays_positive_where_lax_wendroff_undershoots():
    # With the recombination-bound dt the Courant number is small; the
    # upwind weights are all non-negative (6 s + c <= 1) and the explicit
    # recombination factor 1 - alpha dt n stays positive (alpha dt n <= 0.5),
    # so densities stay >= 0.  Lax-Wendroff at the same dt undershoots below
    # zero next to the sharp tracks (the source of its divergence at high LET).
    nx, nz, dx, V = 24, 40, 5e-4, 260.0
    tr = synth.uniform_tracks(99, 40, nx * dx, nx * dx, 1.2e-3, let=740.0)
    mins = {}
    for sch in (o.SCHEME_UPWIND, o.SCHEME_LAX_WENDROFF):
        probe = o.Oracle(nx, nx, nz, dx, 1e-12, voltage_V=V)
        probe.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        npk = max(probe.density(0).max(), probe.density(1).max())
        dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, scheme=sch)
        O = o.Oracle(nx, nx, nz, dx, dt, voltage_V=V, scheme=sch)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        lo = np.inf
        for _ in range(6):
            O.step(20)
            lo = min(lo, O.density(0).min(), O.density(1).min())
        mins[sch] = lo
    assert mins[o.SCHEME_UPWIND] >= 0.0
    assert mins[o.SCHEME_LAX_WENDROFF] < 0.0


# --------------------------------------------------------------------------
# continuous beam: steady-state efficiency of the ions that left the domain
# --------------------------------------------------------------------------
def test_steady_state_of_a_sparse_track_train_is_the_single_track_f():
    # Tracks of one LET at one position, P steps apart, with P longer than a
    # track's life: no two tracks share the domain, so over any window of P
    # steps the ions that leave are exactly one track's ions, and the window
    # efficiency dCol / (dCol + 2 dRec + dLost) must equal the single-track f
    # (collected / released at completion).  Counting the released ions of the
    # window instead, or a recombined pair as one ion, breaks the equality.
    nx, ny, nz, dx, V = 16, 16, 20, 5e-4, 300.0
    kw = dict(mu=MU, D=DD, alpha=ALPHA, voltage_V=V, lateral_bc=o.LATERAL_ABSORBING, scheme=o.SCHEME_UPWIND)
    let, b = 300.0, 1e-3
    dt = o.dt_rule(dx, V, nz * dx, n_peak=o.peak_track_density([let], [b]), scheme=o.SCHEME_UPWIND)
    P = 400
    one = o.Oracle(nx, ny, nz, dx, dt, **kw)
    one.deposit([0.5 * nx * dx], [0.5 * ny * dx], [let], [b])
    one.step(P)
    t1 = one.tallies()
    assert t1.in_domain.sum() / t1.released.sum() < 1e-13      # a track's life is shorter than P
    f1 = t1.f
    assert 0.0 < f1 < 1.0 and t1.recombined > 0 and t1.lost_lateral.sum() > 0
    n = 6
    steps = np.arange(n, dtype=np.int64) * P
    xs, ys = np.full(n, 0.5 * nx * dx), np.full(n, 0.5 * ny * dx)
    train = o.Oracle(nx, ny, nz, dx, dt, **kw)
    r = train.run_to_steady_state(xs, ys, np.full(n, let), np.full(n, b), steps, P, 1e-9, n * P)
    assert r["stop"] == 0 and r["steps"] == 2 * P and r["windows"] == 2
    assert r["f_ss"] == pytest.approx(f1, rel=1e-11)
    assert r["f_window"] == pytest.approx(f1, rel=1e-11)
    # with tol = 0 the rule never holds: all 12 windows run, each holding one
    # track's ions, so every batch has the same efficiency and the batch-means
    # error vanishes
    n = 12
    steps = np.arange(n, dtype=np.int64) * P
    xs, ys = np.full(n, 0.5 * nx * dx), np.full(n, 0.5 * ny * dx)
    train = o.Oracle(nx, ny, nz, dx, dt, **kw)
    r = train.run_to_steady_state(xs, ys, np.full(n, let), np.full(n, b), steps, P, 0.0, n * P)
    assert r["stop"] == 1 and r["windows"] == n
    assert r["f_ss"] == pytest.approx(f1, rel=1e-11)
    assert r["f_ss_stderr"] < 1e-12
    assert r["released"] == pytest.approx(n * t1.released.sum(), rel=1e-12)
    assert r["departed"] == pytest.approx(r["released"], rel=1e-9)


def test_steady_state_runner_does_not_stop_on_idle_windows():
    # One track, then nothing: once it has left, every window is idle and the
    # aggregate no longer moves.  An idle window carries no departures, so it
    # is not judged and the run ends at the step limit (a rule that judged it
    # would call this steady after the track's life).
    nx, nz, dx, V, let, b = 16, 20, 5e-4, 300.0, 300.0, 1e-3
    kw = dict(mu=MU, D=DD, alpha=ALPHA, voltage_V=V, lateral_bc=o.LATERAL_ABSORBING, scheme=o.SCHEME_UPWIND)
    dt = o.dt_rule(dx, V, nz * dx, n_peak=o.peak_track_density([let], [b]), scheme=o.SCHEME_UPWIND)
    O = o.Oracle(nx, nx, nz, dx, dt, **kw)
    r = O.run_to_steady_state([0.5 * nx * dx], [0.5 * nx * dx], [let], [b], np.zeros(1, dtype=np.int64),
                              100, 1e-3, 1200)
    assert r["stop"] == 1 and r["windows"] == 12
    assert 0.0 < r["f_ss"] < 1.0


def test_steady_state_runner_stops_at_the_step_limit():
    # a window longer than the limit: no window runs, the limit is reported
    O = o.Oracle(8, 8, 8, 5e-4, 1e-9, mu=MU, D=DD, alpha=ALPHA, voltage_V=100.0)
    r = O.run_to_steady_state([], [], [], [], np.zeros(0, dtype=np.int64), 50, 1e-5, 40)
    assert r["stop"] == 1 and r["steps"] == 0 and r["windows"] == 0 and math.isnan(r["f_ss"])


def test_ratio_batch_stderr_reduces_to_the_standard_error_of_a_mean():
    # with equal window weights the ratio estimator is the mean of the window
    # values, and its batch-means error (one window per batch) is the
    # textbook s / sqrt(n): values alternating 0.1, 0.3 have s = sqrt(0.1/9)
    se = o.ratio_batch_stderr([0.1, 0.3] * 5, [1.0] * 10)
    assert se == pytest.approx(math.sqrt(0.1 / 9.0) / math.sqrt(10.0), rel=1e-14)
    # proportional windows give zero; fewer than 10 windows give NaN
    assert o.ratio_batch_stderr([0.2 * k for k in range(1, 21)], [float(k) for k in range(1, 21)]) < 1e-15
    assert math.isnan(o.ratio_batch_stderr([0.1] * 9, [1.0] * 9))
    # batches of two windows: sums per batch
    c = [0.1, 0.1, 0.3, 0.3] * 5
    assert o.ratio_batch_stderr(c, [1.0] * 20) == pytest.approx(
        math.sqrt(10.0 / 9.0 * 10 * 0.2 ** 2) / 20.0, rel=1e-14)


# --------------------------------------------------------------------------
# space-charge term of Eq. (theEquation): -/+ mu n div E, div E = q/eps0 (n+ - n-)
# --------------------------------------------------------------------------
Q_EPS0 = 1.602176634e-19 / 8.8541878128e-14   # retyped from CODATA, not from the oracle


@pytest.mark.parametrize("species", [0, 1])
def test_space_charge_of_a_lone_species_follows_its_recurrence(species):
    # One species, uniform, no field, no diffusion, no recombination: each
    # cell obeys n <- n - dt mu q/eps0 n^2 exactly (the cloud repels itself;
    # for n- the sign of the term and of div E both flip), tending to
    # n0 / (1 + mu q/eps0 n0 t).  A wrong sign, species or coefficient fails.
    n0, dt, steps = 4e12, 2e-10, 40
    mu = MU[species]
    O = o.Oracle(3, 3, 3, 5e-4, dt, mu=MU, D=(0.0, 0.0), alpha=0.0, voltage_V=0.0, space_charge=True)
    f = np.full((3, 3, 3), n0)
    z = np.zeros((3, 3, 3))
    O.set_density(f, z) if species == 0 else O.set_density(z, f)
    n = n0
    for _ in range(steps):
        n = n - dt * mu * Q_EPS0 * n * n
    O.step(steps)
    got = O.density(species)
    assert np.allclose(got, n, rtol=1e-13, atol=0)
    assert np.all(O.density(1 - species) == 0.0)
    t = O.tallies()
    vol = (5e-4) ** 3 * 27
    assert t.space_charge[species] == pytest.approx((n - n0) * vol, rel=1e-12)
    cont = n0 / (1.0 + mu * Q_EPS0 * n0 * dt * steps)
    assert n == pytest.approx(cont, rel=0.1) and abs(n - cont) / n0 < mu * Q_EPS0 * n0 * dt * 2


def test_space_charge_leaves_a_neutral_plasma_alone():
    # n+ = n- everywhere: div E = 0, so with no transport and no recombination
    # nothing changes, bitwise
    O = o.Oracle(3, 3, 3, 5e-4, 1e-9, mu=MU, D=(0.0, 0.0), alpha=0.0, voltage_V=0.0, space_charge=True)
    f = np.full((3, 3, 3), 3e12)
    O.set_density(f, f)
    O.step(10)
    assert np.array_equal(O.density(0), f) and np.array_equal(O.density(1), f)
    assert np.all(O.tallies().space_charge == 0.0)


def test_space_charge_conservation_and_proton_invariance():
    # With the term on, the balance closes with its tally:
    # released + added = in domain + collected + lost + recombined.  At a
    # proton-like LET the term changes f by less than 1e-4 (Sec. Conclusions: negligible for protons).
    nx, ny, nz, dx, V = 16, 16, 20, 5e-4, 200.0
    for let, check_f in ((300.0, False), (2e-3, True)):
        npk = o.peak_track_density([let], [1e-3])
        dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, scheme=o.SCHEME_UPWIND, space_charge=True)
        fs = []
        for sc in (True, False):
            O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V,
                         lateral_bc=o.LATERAL_ABSORBING, scheme=o.SCHEME_UPWIND, space_charge=sc)
            O.deposit([0.5 * nx * dx], [0.5 * ny * dx], [let], [1e-3])
            O.step(150)
            t = O.tallies()
            for s in range(2):
                lhs = t.released[s] + t.space_charge[s]
                rhs = t.in_domain[s] + t.collected[s] + t.lost_lateral[s] + t.recombined
                assert lhs == pytest.approx(rhs, rel=1e-12)
            if sc and not check_f:
                assert t.space_charge[0] < 0 and abs(t.space_charge[0]) > 1e-6 * t.released[0]
            fs.append(t.f)
        if check_f:
            assert abs(fs[0] - fs[1]) < 1e-4


# ---------------------------------------------------------------------------
# the doubling step-size ladder of a run to completion
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("space_charge", [False, True])
def test_ladder_rung_is_the_largest_admissible_power_of_two(space_charge):
    # By enumeration: the rung is min(cap, dt 2^j) for the largest j with
    # every bound held at dt 2^j, and never below dt.
    rng = np.random.default_rng(17)
    mu_max = max(MU)
    for _ in range(3000):
        dt = 10.0 ** rng.uniform(-10, -6)
        nmax = 10.0 ** rng.uniform(7, 15) * rng.choice([1.0, 1.0, 0.0])
        kappa = float(rng.choice([0.5, 0.25, 0.1]))
        cap = dt * 10.0 ** rng.uniform(-0.5, 4.0)

        def ok(r):
            return ALPHA * r * nmax <= kappa and (not space_charge or mu_max * o.Q_OVER_EPS0 * r * nmax <= kappa)
        js = [j for j in range(1, 80) if ok(dt * 2.0 ** j)]
        want = dt if not js else max(dt, min(cap, dt * 2.0 ** max(js)))
        assert o.ladder_dt(dt, nmax, ALPHA, cap, kappa, mu_max, space_charge) == want


def test_ladder_on_a_uniform_plasma_follows_the_scalar_recurrence():
    # No transport (V = 0, D = 0): every cell obeys n <- n - alpha dt n^2 with
    # the dt each check picks; the simulated time is the sum of the dt; the
    # rung rises as the plasma thins (n ~ 1/(alpha t)).  Against the continuum
    # n0/(1 + alpha n0 t): a step raises 1/n by alpha dt/(1 - h) with
    # h = alpha dt n <= kappa, i.e. by between alpha dt and alpha dt/(1 - kappa),
    # so (1 - kappa) n_exact <= n <= n_exact whatever the rungs.
    n0, kappa = 4e12, 0.25
    O = o.Oracle(3, 3, 3, 5e-4, kappa / (ALPHA * n0), mu=MU, D=(0.0, 0.0), alpha=ALPHA, voltage_V=0.0)
    f = np.full((3, 3, 3), n0)
    O.set_density(f, f)
    n, t, rungs = n0, 0.0, []
    for _ in range(14):
        tt = O.tallies()
        nmax = float(max(tt.n_max))
        dt = o.ladder_dt(O.dt, nmax, ALPHA, math.inf, kappa)
        assert ALPHA * dt * nmax <= kappa < ALPHA * (2.0 * dt) * nmax or dt == O.dt
        O.set_dt(dt)
        rungs.append(dt)
        O.step(4)
        for _ in range(4):
            n = n - ALPHA * dt * n * n
            t += dt
    for s in range(2):
        np.testing.assert_allclose(O.density(s), n, rtol=1e-14, atol=0)
    assert O.tallies().t_s == pytest.approx(t, rel=1e-14)
    assert all(b >= a for a, b in zip(rungs, rungs[1:])) and rungs[-1] >= 16 * rungs[0]
    exact = n0 / (1.0 + ALPHA * n0 * t)
    assert (1.0 - kappa) * exact <= n <= exact
    assert n < 0.95 * exact   # the rungs sit at the bound, so the lag is not negligible


def _dense_pulse():
    nx, ny, nz, dx, V = 24, 24, 40, 5e-4, 50.0
    tr = synth.uniform_tracks(11, 6, nx * dx, ny * dx, 1e-3, let="loguniform")
    tr.let_keV_um[:] = np.maximum(tr.let_keV_um, 100.0)
    return nx, ny, nz, dx, V, tr


def test_ladder_cuts_the_steps_of_a_dense_pulse_and_keeps_f():
    # Six tracks of 100-720 keV/um at 50 V (upwind drift, which keeps the
    # densities non-negative): the fixed step is bound by recombination at
    # the track cores; the ladder lets it rise to the Eq. (vNeum) step as the
    # cores recombine.  Measured: 1600 fixed steps against 192, f 0.10467
    # against 0.10389 (the fixed-step f at kappa -> 0 is about 0.1057).
    nx, ny, nz, dx, V, tr = _dense_pulse()
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
    dt0 = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, scheme=o.SCHEME_UPWIND)
    cap = o.dt_von_neumann(dx, V, nz * dx, MU, DD, o.SCHEME_UPWIND)
    out = {}
    for ladder in (False, True):
        O = o.Oracle(nx, ny, nz, dx, dt0, mu=MU, D=DD, alpha=ALPHA, voltage_V=V, scheme=o.SCHEME_UPWIND)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        steps, done, log = O.run_to_completion(1e-6, 100_000, 64, ladder=ladder)
        assert done
        t = O.tallies()
        out[ladder] = (steps, t.f, log, t)
        # the charge balance holds whatever the step sequence
        for s in range(2):
            rhs = t.in_domain[s] + t.collected[s] + t.lost_lateral[s] + t.recombined
            assert rhs == pytest.approx(t.released[s], rel=1e-12)
    steps_f, f_f, _, _ = out[False]
    steps_l, f_l, log, t = out[True]
    assert 5 * steps_l <= steps_f
    assert abs(f_l - f_f) < 2e-3
    # the log: the rung rises, stays within the bounds it was decided on, ends
    # at the Eq. (vNeum) step, and the time is the sum of the steps' dt
    dts = [e[1] for e in log]
    assert dts[0] == dt0 and all(b > a for a, b in zip(dts, dts[1:]))
    for step, dt, nmax in log[1:]:
        assert dt <= cap and (ALPHA * dt * nmax <= 0.5)
    assert dts[-1] == cap
    edges = [e[0] for e in log] + [steps_l]
    assert t.t_s == pytest.approx(sum(d * (b - a) for d, a, b in zip(dts, edges, edges[1:])), rel=1e-13)


# ---------------------------------------------------------------------------
# tracks at an angle to the field (Fig. setup (a), Eq. angle)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lat", [o.LATERAL_PERIODIC, o.LATERAL_ABSORBING])
def test_angled_deposit_at_zero_is_the_parallel_deposit(lat):
    nx, ny, nz, dx = 40, 30, 50, 2e-4
    A = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=lat)
    P = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=lat)
    xs, ys, lets, bs = [0.0041, 0.0002], [0.0033, 0.0057], [50.0, 3.0], [1e-3, 6e-4]
    ra = A.deposit(xs, ys, lets, bs)
    rb = P.deposit_angled(xs, ys, lets, bs, [0.0, 0.0])
    for s in range(2):
        assert np.array_equal(A.density(s), P.density(s))
    assert rb == pytest.approx(ra, rel=1e-13)


@pytest.mark.parametrize("theta", [0.3, 0.8, 1.2, math.pi / 2])
def test_angled_deposit_releases_n0_times_the_path_length(theta):
    # Periodic faces, whole windows: every plane holds N0 dz / cos(theta)
    # (Eq. created along the tilted path); parallel to the electrodes the
    # track crosses the box along x, N0 Lx (the Gaussian in z sampled at the
    # cell centres, dz = b/5, sums to its integral far below 1e-10).
    nx, ny, nz, dx = 40, 30, 50, 2e-4
    O = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=o.LATERAL_PERIODIC)
    N0 = 50.0 * 1e7 / 34.0
    r = O.deposit_angled([0.0041], [0.0033], [50.0], [1e-3], [theta])
    want = N0 * nx * dx if theta == math.pi / 2 else N0 * nz * dx / math.cos(theta)
    assert r == pytest.approx(want, rel=1e-10)
    assert O.density(0).sum() * dx ** 3 == pytest.approx(r, rel=1e-12)


def test_angled_deposit_planes_shift_by_dz_tan_theta_and_widen_by_one_over_cos():
    # In each z plane the track's cross-section is the Gaussian of width
    # b/cos(theta) along x, centred where the axis crosses the plane:
    # x0 + (z_k - d/2) tan(theta).  Cell averages keep its mean exactly and
    # add dx^2/12 to its variance b^2/(2 cos^2) (absorbing faces, the whole
    # cross-section inside the box).
    nx, ny, nz, dx, b, th = 120, 40, 20, 2e-4, 1e-3, 0.5
    O = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=o.LATERAL_ABSORBING)
    x0, y0 = 0.5 * nx * dx, 0.5 * ny * dx
    O.deposit_angled([x0], [y0], [10.0], [b], [th])
    n = O.density(0)
    xc = (np.arange(nx) + 0.5) * dx
    for k in range(nz):
        px = n[k].sum(axis=0)
        mean = (px * xc).sum() / px.sum()
        var = (px * (xc - mean) ** 2).sum() / px.sum()
        zk = (k + 0.5) * dx
        assert mean == pytest.approx(x0 + (zk - 0.5 * nz * dx) * math.tan(th), abs=1e-9 * dx)
        assert var == pytest.approx(b * b / (2 * math.cos(th) ** 2) + dx * dx / 12, rel=1e-9)


def test_track_parallel_to_the_electrodes_follows_jaffe_angle():
    # Eq. (angle) at theta = pi/2: a track along x at mid-gap (periodic x, so
    # it is infinite), LET 1 keV/um, b = 10 um, E = 1000 V/cm (Z = 591, deep
    # in the large-angle, large-Z regime where the approximation holds).
    # Measured: f - f_J = -2.34e-3 at dx = b/5 and -7.0e-4 at b/10
    # (1 - f_J = 0.0254); the gap closes as the grid resolves the column.
    b, E, let = 1e-3, 1000.0, 1.0
    fj = o.jaffe_angle(let, b, E, math.pi / 2, 0.5 * (MU[0] + MU[1]), 0.037, ALPHA)
    gaps = []
    for frac in (5, 10):
        dx = b / frac
        nx, ny, nz = 4, 10 * frac, 40 * frac
        V = E * nz * dx
        dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=o.peak_track_density([let], [b]))
        O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V)
        O.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [let], [b], [math.pi / 2])
        _, done, _ = O.run_to_completion(1e-6, 100_000, 64)
        assert done
        gaps.append(abs(O.tallies().f - fj))
    assert gaps[0] < 3e-3 and gaps[1] < 1e-3 and gaps[1] < gaps[0]


def test_run_to_completion_stops_on_a_state_that_is_not_finite():
    # Lax-Wendroff at the recombination-bound step on a dense pulse diverges:
    # at the small Courant number its undershoots make -alpha n+ n- a
    # source.  The run must stop at the first check that sees it, as the
    # library's IT_EUNSTABLE does, not step on to max_steps.
    nx, ny, nz, dx, V = 24, 24, 40, 5e-4, 50.0
    tr = synth.uniform_tracks(11, 6, nx * dx, ny * dx, 1e-3, let="loguniform")
    tr.let_keV_um[:] = np.maximum(tr.let_keV_um, 100.0)
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
    dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, kappa=0.25)
    O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V)
    O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
    with pytest.raises(FloatingPointError):
        O.run_to_completion(1e-6, 200_000, 64)
    assert O.tallies().steps < 5000


def test_angled_deposit_is_continuous_across_the_parallel_to_electrodes_switch():
    # Absorbing faces, so a tilted track has no periodic images: just above
    # and just below cos(theta) dx / b = 1e-3 the erf form and the
    # cell-centre form describe the same single column (its x profile is
    # b/cos = 200 b wide, nearly flat across the box).  The midpoint rule
    # differs from the cell integral by about (cos dx/b)^2/24 relative and
    # the angles by 1e-6 relative in cos, both far below 1e-6.  (With
    # periodic faces the erf form would sum the images of the tilted track,
    # a stack of parallel tracks, while the near-parallel form is one track
    # by definition.)
    nx, ny, nz, dx, b = 8, 30, 40, 2e-4, 1e-3
    c_switch = 1e-3 * b / dx
    out = []
    for c in (c_switch * (1 + 1e-6), c_switch * (1 - 1e-6)):
        O = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=o.LATERAL_ABSORBING)
        O.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [5.0], [b], [math.acos(c)])
        out.append(O.density(0))
    scale = np.max(out[1])
    assert scale > 0
    assert np.max(np.abs(out[0] - out[1])) <= 1e-6 * scale
