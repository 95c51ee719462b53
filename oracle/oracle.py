"""FP64 CPU oracle for the IonTracks transport step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never touches the CUDA library and
the CUDA library never touches it.

Contents
--------
* ``Oracle`` -- ctypes handle on ``liboracle.so`` (plain C, FP64): deposition
  (Eqs. linear_density, Gaussian, created), the explicit step of
  Eq. (theEquation) discretised as in the Appendix, electrode / lateral
  collection tallies and f (Eq. collection_efficiency).
* ``dt_von_neumann`` -- the largest dt allowed by Eq. (vNeum), for both species.
* ``dt_rule`` -- that bound combined with a recombination bound
  kappa / (alpha n_peak); the paper states no bound for the reaction term, so
  this is a reading (explicit Euler on dn/dt = -alpha n^2 is stable only for
  alpha dt n < 2; kappa = 0.5 keeps it monotone).
* ``ladder_dt`` and ``Oracle.run_to_completion(ladder=True)`` -- the same
  bound applied at every completion check to the state's current peak density,
  raising dt by powers of two up to the Eq. (vNeum) step (a reading: the
  densest cells, which set the initial bound, recombine first).
* Closed forms used as pins: ``ei`` (exponential integral of the Jaffe
  section, own series/asymptotic code), ``jaffe_parallel`` (Eq. Jaffe_noangle),
  ``jaffe_angle`` (Eq. angle), ``boag_2vm`` (the p = 0 limit of the Boag
  models, f = ln(1+u)/u), ``gaussian_track_diffused`` (Eq. Gaussian under pure
  diffusion, b^2 -> b^2 + 4 D t).

Parity of every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

LATERAL_PERIODIC = 0
LATERAL_ABSORBING = 1
SCHEME_LAX_WENDROFF = 0
SCHEME_UPWIND = 1

EULER_GAMMA = 0.57721566490153286060651209008240243


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d, i, p, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_create.restype = p
        lib.orc_create.argtypes = [i, i, i, d, d, d, d, d, d, d, d, i, i]
        lib.orc_destroy.argtypes = [p]
        lib.orc_deposit.restype = d
        lib.orc_deposit.argtypes = [p, i64, dp, dp, dp, dp, d]
        lib.orc_step.argtypes = [p]
        lib.orc_steps.argtypes = [p, i64]
        lib.orc_in_domain.argtypes = [p, dp, dp]
        lib.orc_tallies.argtypes = [p, dp]
        lib.orc_get_density.argtypes = [p, i, dp]
        lib.orc_set_density.argtypes = [p, dp, dp]
        lib.orc_set_space_charge.argtypes = [p, i]
        lib.orc_space_charge.argtypes = [p, dp]
        lib.orc_deposit_angled.argtypes = [p, i64, dp, dp, dp, dp, dp, d]
        lib.orc_deposit_angled.restype = d
        lib.orc_set_dt.argtypes = [p, d]
        lib.orc_set_dt.restype = ctypes.c_int
        lib.orc_time.argtypes = [p]
        lib.orc_time.restype = d
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Tallies:
    released: np.ndarray        # [2] ions, positive / negative
    collected_anode: np.ndarray
    collected_cathode: np.ndarray
    lost_lateral: np.ndarray
    in_domain: np.ndarray
    recombined: float
    steps: int
    n_min: np.ndarray
    n_max: np.ndarray
    space_charge: np.ndarray = None   # [2] ions added by the space-charge term (negative: removed)
    t_s: float = 0.0                  # simulated time, the sum of every step's dt
    dt_s: float = 0.0                 # the current time step

    @property
    def collected(self) -> np.ndarray:
        return self.collected_anode + self.collected_cathode

    @property
    def f(self) -> float:
        """Eq. (collection_efficiency): ions collected over ions released,
        both species together (reading: f counts the two species' ions)."""
        rel = float(self.released.sum())
        return float(self.collected.sum()) / rel if rel > 0 else float("nan")


class Oracle:
    """One FP64 simulation on the host.  Units are CGS: cm, s, V, ions/cm^3."""

    def __init__(self, nx, ny, nz, dx_cm, dt_s, mu=(1.73, 1.87), D=(0.037, 0.037),
                 alpha=1.6e-6, voltage_V=200.0, lateral_bc=LATERAL_PERIODIC,
                 scheme=SCHEME_LAX_WENDROFF, W_eV=34.0, space_charge=False):
        lib = _load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dt = float(dx_cm), float(dt_s)
        self.gap = self.nz * self.dx
        self.E = float(voltage_V) / self.gap
        self.W = float(W_eV)
        self.V, self.mu, self.D = float(voltage_V), (float(mu[0]), float(mu[1])), (float(D[0]), float(D[1]))
        self.alpha, self.scheme, self.space_charge = float(alpha), int(scheme), bool(space_charge)
        self._h = lib.orc_create(self.nx, self.ny, self.nz, self.dx, self.dt,
                                 float(mu[0]), float(mu[1]), float(D[0]), float(D[1]),
                                 float(alpha), self.E, int(lateral_bc), int(scheme))
        if not self._h:
            raise ValueError("oracle: invalid grid or step")
        lib.orc_set_space_charge(self._h, 1 if space_charge else 0)

    def close(self):
        if self._h:
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def deposit(self, x_cm, y_cm, let_keV_um, b_cm) -> float:
        x = np.ascontiguousarray(x_cm, dtype=np.float64)
        y = np.ascontiguousarray(y_cm, dtype=np.float64)
        L = np.ascontiguousarray(let_keV_um, dtype=np.float64)
        b = np.ascontiguousarray(b_cm, dtype=np.float64)
        n = x.size
        if not (y.size == n and L.size == n and b.size == n):
            raise ValueError("track arrays differ in length")
        if n == 0:
            return 0.0
        return _load().orc_deposit(self._h, n, _dptr(x), _dptr(y), _dptr(L), _dptr(b), self.W)

    def deposit_angled(self, x_cm, y_cm, let_keV_um, b_cm, theta_rad) -> float:
        """Tracks at angle theta in [0, pi/2] to the field, rotated in the x-z
        plane, axes through (x, y, d/2) (Fig. setup (a)); see
        orc_deposit_angled.  Returns the released ions per species."""
        arrs = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64)
                for a in (x_cm, y_cm, let_keV_um, b_cm, theta_rad)]
        n = arrs[0].size
        if any(a.size != n for a in arrs):
            raise ValueError("track arrays differ in length")
        if n == 0:
            return 0.0
        return _load().orc_deposit_angled(self._h, n, *[_dptr(a) for a in arrs], self.W)

    def step(self, n: int = 1):
        _load().orc_steps(self._h, int(n))

    def set_dt(self, dt_s: float):
        """Time step of the steps that follow."""
        if _load().orc_set_dt(self._h, float(dt_s)) != 0:
            raise ValueError("oracle: dt must be positive")
        self.dt = float(dt_s)

    def run_to_completion(self, tol=1e-6, max_steps=10_000_000, check_every=64, ladder=False, kappa=0.5,
                          cfl_safety=1.0):
        """Step until the tracks are dragged apart (end of Sec.
        Implementation): at every check (the first before any step, then every
        check_every steps) stop when the ions left in the domain are below
        tol of the released ones (or nothing was released).  With
        ladder=True each check first raises dt by ladder_dt from the state's
        peak density, capped at cfl_safety times the Eq. (vNeum) step.

        Returns (steps taken, completed, log) where log lists
        (step, dt, n_max) for the initial dt and every change.  Raises
        FloatingPointError when a check finds the state not finite (the
        library's IT_EUNSTABLE), rather than stepping on to max_steps."""
        start = self.tallies().steps
        log = [(start, self.dt, float("nan"))]
        cap = cfl_safety * dt_von_neumann(self.dx, self.V, self.gap, self.mu, self.D, self.scheme)
        while True:
            t = self.tallies()
            rel = float(t.released.sum())
            if not math.isfinite(float(t.in_domain.sum()) + t.recombined):
                raise FloatingPointError(f"oracle: state is not finite at step {t.steps}")
            if rel > 0 and float(t.in_domain.sum()) / rel < tol:
                return t.steps - start, True, log
            if rel == 0:
                return t.steps - start, True, log
            left = start + max_steps - t.steps
            if left <= 0:
                return t.steps - start, False, log
            if ladder:
                nmax = float(max(t.n_max[0], t.n_max[1]))
                nd = ladder_dt(self.dt, nmax, self.alpha, cap, kappa, max(self.mu), self.space_charge)
                if nd > self.dt:
                    self.set_dt(nd)
                    log.append((t.steps, nd, nmax))
            self.step(min(check_every, left))

    def run_schedule(self, x_cm, y_cm, let, b, step_idx, n_steps: int, start_step: int = 0):
        """Deposit each track at the start of its arrival step, then step."""
        step_idx = np.asarray(step_idx, dtype=np.int64)
        order = np.argsort(step_idx, kind="stable")
        xs, ys = np.asarray(x_cm)[order], np.asarray(y_cm)[order]
        Ls, bs, ss = np.asarray(let)[order], np.asarray(b)[order], step_idx[order]
        ptr = int(np.searchsorted(ss, start_step, side="left"))
        for l in range(start_step, start_step + n_steps):
            hi = int(np.searchsorted(ss, l, side="right"))
            if hi > ptr:
                self.deposit(xs[ptr:hi], ys[ptr:hi], Ls[ptr:hi], bs[ptr:hi])
                ptr = hi
            self.step(1)

    def run_to_steady_state(self, x_cm, y_cm, let, b, step_idx, window: int, tol: float, max_steps: int):
        """Continuous beam to steady state (Sec. Implementation, "Distribution
        of ion tracks"), reading "f stable to tol over a window of steps" on
        the ions that have left the domain since the call began: windows of
        `window` steps with the scheduled arrivals; after window w the
        aggregate efficiency is F_w = Col / (Col + 2 Rec + Lost), both
        species, Col collected at the electrodes, Rec recombined pairs (two
        ions each), Lost through absorbing faces, all counted since the call
        began.  The run stops after the first window w >= 2 with
        |F_w - F_{w-1}| < tol that is judged: the window's own departures
        are positive and at least half of (ions released since the call
        began) / w, and the departures since the call began are at least
        half of those released.  Otherwise it ends when the next window would
        pass max_steps.

        Returns a dict: f_ss (= F of the last window), f_ss_stderr (ratio
        estimator over 10 batches of consecutive windows, NaN below 10
        windows), f_window (the last window's own Col / departed), departed,
        released, windows, steps, stop (0 steady, 1 step limit)."""
        def state(t):
            return float(t.collected.sum()), float(t.recombined), float(t.lost_lateral.sum()), float(t.released.sum())

        t = self.tallies()
        start = t.steps
        c_s, r_s, l_s, rel_s = state(t)
        per_window = []                       # (collected, departed) in each window
        prev = (c_s, r_s, l_s)
        F_prev = F = f_win = float("nan")
        C = G = Rel = 0.0
        stop = 1
        while self.tallies().steps - start + window <= max_steps:
            self.run_schedule(x_cm, y_cm, let, b, step_idx, window, start_step=self.tallies().steps)
            c1, r1, l1, rel1 = state(self.tallies())
            dc, dr, dl = c1 - prev[0], r1 - prev[1], l1 - prev[2]
            prev = (c1, r1, l1)
            g = dc + 2.0 * dr + dl
            per_window.append((dc, g))
            f_win = dc / g if g != 0.0 else float("nan")
            C = c1 - c_s
            G = C + 2.0 * (r1 - r_s) + (l1 - l_s)
            Rel = rel1 - rel_s
            F = C / G if G != 0.0 else float("nan")
            w = len(per_window)
            judged = g > 0.0 and g >= 0.5 * Rel / w and G >= 0.5 * Rel
            if judged and w >= 2 and math.isfinite(F) and math.isfinite(F_prev) and abs(F - F_prev) < tol:
                stop = 0
                break
            F_prev = F
        se = ratio_batch_stderr([p[0] for p in per_window], [p[1] for p in per_window])
        return {"f_ss": F, "f_ss_stderr": se, "f_window": f_win, "departed": G, "released": Rel,
                "windows": len(per_window), "steps": self.tallies().steps - start, "stop": stop}

    def tallies(self) -> Tallies:
        lib = _load()
        t = np.zeros(10)
        lib.orc_tallies(self._h, _dptr(t))
        ind = np.zeros(2)
        mm = np.zeros(4)
        lib.orc_in_domain(self._h, _dptr(ind), _dptr(mm))
        sc = np.zeros(2)
        lib.orc_space_charge(self._h, _dptr(sc))
        return Tallies(released=t[0:2].copy(), collected_anode=t[2:4].copy(),
                       collected_cathode=t[4:6].copy(), lost_lateral=t[6:8].copy(),
                       in_domain=ind, recombined=float(t[8]), steps=int(t[9]),
                       n_min=mm[[0, 2]].copy(), n_max=mm[[1, 3]].copy(), space_charge=sc,
                       t_s=float(lib.orc_time(self._h)), dt_s=self.dt)

    def density(self, species: int) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx), dtype=np.float64)
        _load().orc_get_density(self._h, int(species), _dptr(out))
        return out

    def set_density(self, plus: np.ndarray, minus: np.ndarray):
        shape = (self.nz, self.ny, self.nx)
        p = np.ascontiguousarray(np.broadcast_to(plus, shape), dtype=np.float64)
        m = np.ascontiguousarray(np.broadcast_to(minus, shape), dtype=np.float64)
        _load().orc_set_density(self._h, _dptr(p), _dptr(m))


def ratio_batch_stderr(c, g, nb: int = 10) -> float:
    """Standard error of the ratio F = sum(c) / sum(g) of per-window sums by
    batch means: the windows are cut into nb batches of consecutive windows
    (batch k holds windows [k n / nb, (k+1) n / nb)), and with the batch sums
    C_k, G_k and residuals e_k = C_k - F G_k (which sum to zero),
    SE = sqrt(nb / (nb - 1) * sum e_k^2) / sum(g) -- the delta-method error of
    a ratio estimator.  NaN below nb windows or when sum(g) is 0."""
    n = len(c)
    G = float(sum(g))
    if n < nb or G == 0.0:
        return float("nan")
    F = float(sum(c)) / G
    resid = []
    for k in range(nb):
        lo, hi = k * n // nb, (k + 1) * n // nb
        resid.append(float(sum(c[lo:hi])) - F * float(sum(g[lo:hi])))
    return math.sqrt(nb / (nb - 1) * sum(e * e for e in resid)) / G


# ---------------------------------------------------------------------------
# time-step rules
# ---------------------------------------------------------------------------

def dt_von_neumann(dx_cm, voltage_V, gap_cm, mu=(1.73, 1.87), D=(0.037, 0.037),
                   scheme=SCHEME_LAX_WENDROFF) -> float:
    """Largest dt satisfying Eq. (vNeum) for both species with E along z only.

    With dx = dy = dz and s = D dt/dx^2, c = mu E dt/dx the first condition
    reads 6 s + c^2 <= 1, a quadratic in dt; the second, c_x^2 c_y^2 c_z^2 <=
    8 s_x s_y s_z, holds trivially because c_x = c_y = 0.  For the pure upwind
    option the matching bound is 6 s + c <= 1.
    """
    E = voltage_V / gap_cm
    best = math.inf
    for m, d in zip(mu, D):
        a = (m * E / dx_cm) ** 2           # coefficient of dt^2 in c^2
        q = 6.0 * d / dx_cm ** 2           # coefficient of dt in 2(sx+sy+sz)
        v = m * E / dx_cm
        if scheme == SCHEME_UPWIND:
            dt = 1.0 / (q + v) if (q + v) > 0 else math.inf
        elif a > 0:
            dt = (-q + math.sqrt(q * q + 4.0 * a)) / (2.0 * a)
        else:
            dt = 1.0 / q if q > 0 else math.inf
        best = min(best, dt)
    return best


def peak_track_density(let_keV_um, b_cm, W_eV=34.0) -> float:
    """Largest centre density N0/(pi b^2) over a set of tracks (Eq. Gaussian)."""
    let = np.atleast_1d(np.asarray(let_keV_um, dtype=np.float64))
    b = np.atleast_1d(np.asarray(b_cm, dtype=np.float64))
    if let.size == 0:
        return 0.0
    N0 = let * 1e7 / W_eV
    return float(np.max(N0 / (math.pi * b * b)))


# Elementary charge (C) over the vacuum permittivity (F/cm), V cm: the
# Maxwell-Gauss equation div E = q/eps0 (n+ - n-) with n in ions/cm^3.
Q_OVER_EPS0 = 1.602176634e-19 / 8.8541878128e-14


def dt_rule(dx_cm, voltage_V, gap_cm, mu=(1.73, 1.87), D=(0.037, 0.037), alpha=1.6e-6,
            n_peak=0.0, cfl_safety=1.0, kappa=0.5, scheme=SCHEME_LAX_WENDROFF, space_charge=False) -> float:
    """dt = min(cfl_safety * dt_vN, kappa / (alpha n_peak)), and with the
    space-charge term also kappa / (max(mu) q/eps0 n_peak): the term decays a
    lone species at the rate mu q/eps0 n, resolved the same way as
    recombination."""
    dt = cfl_safety * dt_von_neumann(dx_cm, voltage_V, gap_cm, mu, D, scheme)
    if alpha > 0 and n_peak > 0:
        dt = min(dt, kappa / (alpha * n_peak))
    if space_charge and n_peak > 0:
        dt = min(dt, kappa / (max(mu) * Q_OVER_EPS0 * n_peak))
    return dt


def ladder_dt(dt, n_max, alpha, dt_cap, kappa=0.5, mu_max=0.0, space_charge=False, max_doublings=60) -> float:
    """One check of the doubling step-size ladder (reading: the paper's dt
    rule, Eq. vNeum, covers transport only; the reaction bound of dt_rule is
    set by the densest cells, which recombine first).  Returns
    min(dt_cap, dt 2^j) for the largest j >= 0 with alpha (dt 2^j) n_max <=
    kappa, and with the space-charge term also mu_max q/eps0 (dt 2^j) n_max
    <= kappa; never less than dt (the ladder only rises).  Products are
    formed left to right."""
    def within(r):
        if alpha * r * n_max > kappa:
            return False
        if space_charge and mu_max * Q_OVER_EPS0 * r * n_max > kappa:
            return False
        return True
    r = dt
    for _ in range(max_doublings):
        if not (r < dt_cap and within(2.0 * r)):
            break
        r *= 2.0
    return max(dt, min(r, dt_cap))


# ---------------------------------------------------------------------------
# closed forms (pins)
# ---------------------------------------------------------------------------

def ei_scaled(x: float) -> float:
    """exp(-x) Ei(x) for x > 0, Ei as defined beside Eq. (Jaffe_noangle).

    x <= 40: the convergent series Ei(x) = gamma + ln x + sum x^k/(k k!),
    whose terms are all positive for x > 0.  x > 40: the asymptotic series
    exp(-x) Ei(x) ~ (1/x) sum_k k!/x^k, cut at its smallest term.
    """
    if not x > 0:
        raise ValueError("ei_scaled needs x > 0")
    if x <= 40.0:
        term, s, k = 1.0, 0.0, 1
        while True:
            term *= x / k
            add = term / k
            s += add
            if add < 1e-18 * s:
                break
            k += 1
        return math.exp(-x) * (EULER_GAMMA + math.log(x) + s)
    term, s, k = 1.0, 1.0, 1
    while k < 200:
        nxt = term * k / x
        if nxt >= term:
            break
        term = nxt
        s += term
        k += 1
    return s / x


def ei(x: float) -> float:
    return ei_scaled(x) * math.exp(x)


def jaffe_y(let_keV_um, b_cm, gap_cm, E_V_cm, mu_mean, D_mean, alpha, W_eV=34.0):
    N0 = let_keV_um * 1e7 / W_eV
    y1 = 8.0 * math.pi * D_mean / (alpha * N0)
    y2 = 2.0 * gap_cm * D_mean / (mu_mean * b_cm ** 2 * E_V_cm)
    return y1, y2


def jaffe_parallel(let_keV_um, b_cm, gap_cm, E_V_cm, mu_mean, D_mean, alpha,
                   W_eV=34.0, method="auto") -> float:
    """Eq. (Jaffe_noangle): f = (y1/y2) e^{-y1} [Ei(y1 + ln(1+y2)) - Ei(y1)].

    ``method='ei'`` evaluates the printed form with ``ei_scaled`` (no
    overflow: e^{-y1} Ei(y1+L) = e^{L} ei_scaled(y1+L)).  ``method='quad'``
    uses the equivalent integral (y1/y2) int_0^{ln(1+y2)} e^g / (y1+g) dg
    (substitute u = y1 + g and use dEi/du = e^u/u) by composite
    Gauss-Legendre on panels that grade geometrically away from g = 0.
    """
    y1, y2 = jaffe_y(let_keV_um, b_cm, gap_cm, E_V_cm, mu_mean, D_mean, alpha, W_eV)
    L = math.log1p(y2)
    if method == "auto":
        method = "ei" if y1 > 1e-3 and L / y1 > 1e-6 else "quad"
    if method == "ei":
        return (y1 / y2) * (math.exp(L) * ei_scaled(y1 + L) - ei_scaled(y1))
    xg, wg = np.polynomial.legendre.leggauss(24)
    edges = [0.0]
    h = min(L, max(y1, 1e-300))
    while edges[-1] + h < L:
        edges.append(edges[-1] + h)
        h *= 2.0
    edges.append(L)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        g = 0.5 * (b - a) * xg + 0.5 * (b + a)
        tot += 0.5 * (b - a) * float(np.sum(wg * np.exp(g) / (y1 + g)))
    return (y1 / y2) * tot


def jaffe_angle(let_keV_um, b_cm, E_V_cm, theta, mu_mean, D_mean, alpha, W_eV=34.0) -> float:
    """Eq. (angle): f = 1/(1 + S(Z)/y1), S(Z) = e^Z (i pi/2) H0^(1)(iZ).

    For real Z > 0, (i pi/2) H0^(1)(iZ) is the modified Bessel function K0(Z),
    so S(Z) = e^Z K0(Z) (scipy.special.k0e)."""
    from scipy.special import k0e
    N0 = let_keV_um * 1e7 / W_eV
    y1 = 8.0 * math.pi * D_mean / (alpha * N0)
    Z = (mu_mean * b_cm * E_V_cm * math.sin(theta) / (2.0 * D_mean)) ** 2
    return 1.0 / (1.0 + float(k0e(Z)) / y1)


def boag_u(alpha, mu_p, mu_m, n_cm3, gap_cm, voltage_V) -> float:
    """u of the Boag models: alpha/(mu+ + mu-) * n d^2 / V."""
    return alpha / (mu_p + mu_m) * n_cm3 * gap_cm ** 2 / voltage_V


def boag_2vm(u: float) -> float:
    """p = 0 limit of Boag's models 1-3: f = ln(1+u)/u."""
    return math.log1p(u) / u if u != 0 else 1.0


def gaussian_track_diffused(r_cm, t_s, N0, b_cm, D) -> np.ndarray:
    """Eq. (Gaussian) after pure 2D diffusion for time t: b^2 -> b^2 + 4 D t."""
    bb = b_cm * b_cm + 4.0 * D * t_s
    return N0 / (math.pi * bb) * np.exp(-np.asarray(r_cm) ** 2 / bb)
