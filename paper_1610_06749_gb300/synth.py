"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only -- none of the method's arithmetic.
Every random draw comes from SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): state +=
0x9E3779B97F4A7C15 and an output mix of two xor-shift-multiply rounds.
A uniform double is (r >> 11) * 2^-53.  Both the oracle and the CUDA path
receive the arrays produced here, so track positions are bit-identical on
the two sides by construction.

Workload recipes follow the paper's physical model (tracks parallel to the
field, uniform irradiation, Poisson arrivals; Sec. "Distribution of ion
tracks") at the grid sizes of the benchmark configurations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for a 64-bit seed (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from SplitMix64: (r >> 11) * 2^-53."""
    r = splitmix64(seed, n)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class TrackList:
    """Tracks parallel to the field that span the gap.

    x_cm, y_cm: centre; let_keV_um: LET; b_cm: Gaussian radius; step: the
    time step at whose start the track is deposited (0 for a single pulse).
    """
    x_cm: np.ndarray
    y_cm: np.ndarray
    let_keV_um: np.ndarray
    b_cm: np.ndarray
    step: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.step is None:
            self.step = np.zeros(self.x_cm.size, dtype=np.int64)

    def __len__(self):
        return int(self.x_cm.size)

    def select(self, mask) -> "TrackList":
        return TrackList(self.x_cm[mask], self.y_cm[mask], self.let_keV_um[mask],
                         self.b_cm[mask], self.step[mask])


def uniform_tracks(seed: int, n: int, Lx_cm: float, Ly_cm: float, b_cm: float,
                   let="loguniform", let_range=(1.0, 1000.0)) -> TrackList:
    """n tracks at uniform (x, y) over [0,Lx) x [0,Ly).

    let='loguniform': LET = lo * (hi/lo)^u; let=<float>: fixed LET;
    let=('mixture', [(LET, weight), ...]): two-or-more-species mixture.
    Draws per track: x, y, LET (three consecutive uniforms).
    """
    u = uniform01(seed, 3 * n).reshape(n, 3) if n > 0 else np.zeros((0, 3))
    x = u[:, 0] * Lx_cm
    y = u[:, 1] * Ly_cm
    L = _let_from_uniform(u[:, 2], let, let_range)
    return TrackList(x, y, L, np.full(n, float(b_cm)))


def _let_from_uniform(u, let, let_range):
    if isinstance(let, str) and let == "loguniform":
        lo, hi = let_range
        return lo * (hi / lo) ** u
    if isinstance(let, tuple) and let[0] == "mixture":
        species = let[1]
        w = np.array([s[1] for s in species], dtype=np.float64)
        cw = np.cumsum(w / w.sum())
        vals = np.array([s[0] for s in species], dtype=np.float64)
        idx = np.searchsorted(cw, u, side="right")
        return vals[np.minimum(idx, len(vals) - 1)]
    return np.full(u.shape, float(let))


def circle_tracks(seed: int, n: int, centre_cm, r_min_cm: float, b_cm: float,
                  let=100.0) -> TrackList:
    """Tracks uniform inside a circle of radius r_min (rejection sampling)."""
    xs, ys = [], []
    k = 0
    while len(xs) < n:
        u = uniform01(seed + 7919 * k, 4 * max(n, 16)).reshape(-1, 2)
        k += 1
        for a, b in u:
            px, py = 2 * a - 1, 2 * b - 1
            if px * px + py * py < 1.0:
                xs.append(centre_cm[0] + r_min_cm * px)
                ys.append(centre_cm[1] + r_min_cm * py)
                if len(xs) == n:
                    break
    L = _let_from_uniform(np.zeros(n), let, (1.0, 1000.0))
    return TrackList(np.array(xs), np.array(ys), L, np.full(n, float(b_cm)))


def poisson_tracks(seed: int, rate_per_cm2_s: float, Lx_cm: float, Ly_cm: float,
                   dt_s: float, n_steps: int, b_cm: float, let) -> TrackList:
    """Poisson arrivals over the section Lx*Ly for n_steps steps of dt.

    Inter-arrival times -ln(1-u)/lambda with lambda = rate * Lx * Ly; a track
    arriving at t is deposited at the start of step floor(t/dt).  Draws per
    track: inter-arrival, x, y, LET (four consecutive uniforms).
    """
    lam = rate_per_cm2_s * Lx_cm * Ly_cm
    T = dt_s * n_steps
    expect = lam * T
    chunk = int(expect + 10 * math.sqrt(expect + 1) + 16)
    u = uniform01(seed, 4 * chunk).reshape(chunk, 4)
    t = np.cumsum(-np.log1p(-u[:, 0]) / lam)
    keep = t < T
    u, t = u[keep], t[keep]
    x = u[:, 1] * Lx_cm
    y = u[:, 2] * Ly_cm
    L = _let_from_uniform(u[:, 3], let, (1.0, 1000.0))
    step = np.floor(t / dt_s).astype(np.int64)
    step = np.minimum(step, n_steps - 1)
    return TrackList(x, y, L, np.full(x.size, float(b_cm)), step)


# ---------------------------------------------------------------------------
# workloads (grid sizes and physical constants of the benchmark configurations)
# ---------------------------------------------------------------------------

AIR = dict(mu=(1.73, 1.87), D=(0.037, 0.037), alpha=1.6e-6, W_eV=34.0)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx_cm: float
    voltage_V: float
    b_cm: float
    precision: str          # "f32" or "f64"
    lateral: str            # "periodic" or "absorbing"
    seed: int
    n_tracks: int = 0
    note: str = ""

    @property
    def gap_cm(self):
        return self.nz * self.dx_cm

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


def single_track_48x48x100() -> Workload:
    """One track along z at the centre: LET 100 keV/um, b = 10 um, dx = 2 um,
    200 V over a 200 um gap, FP64, absorbing lateral faces."""
    return Workload("single_track_48x48x100_fp64", 48, 48, 100, 2e-4, 200.0, 1e-3,
                    "f64", "absorbing", 0, 1)


def single_track_tracks(w: Workload) -> TrackList:
    c = 0.5 * w.nx * w.dx_cm
    return TrackList(np.array([c]), np.array([0.5 * w.ny * w.dx_cm]),
                     np.array([100.0]), np.array([w.b_cm]))


def pulsed_256x256x400(voltage_V: float = 200.0) -> Workload:
    """2000 tracks per pulse at uniform (x, y), log-uniform LET 1-1000 keV/um,
    b = 10 um, dx = 5 um (2 mm gap), FP32, periodic lateral faces."""
    return Workload(f"pulsed_256x256x400_{int(voltage_V)}V_fp32", 256, 256, 400, 5e-4,
                    voltage_V, 1e-3, "f32", "periodic", 1610067490 + int(voltage_V), 2000)


def pulsed_tracks(w: Workload) -> TrackList:
    return uniform_tracks(w.seed, w.n_tracks, w.nx * w.dx_cm, w.ny * w.dx_cm, w.b_cm,
                          let="loguniform", let_range=(1.0, 1000.0))


def continuous_512x512x256() -> Workload:
    """Poisson arrivals, LET mixture 20/200 keV/um at 70/30, b = 10 um,
    dx = 8 um, 300 V, FP32, periodic lateral faces."""
    return Workload("continuous_512x512x256_300V_fp32", 512, 512, 256, 8e-4, 300.0, 1e-3,
                    "f32", "periodic", 1610067491)


CONTINUOUS_LET = ("mixture", [(20.0, 0.7), (200.0, 0.3)])


def batch_descriptors(seed: int = 1610067492, n: int = 256):
    """Independent simulations of uneven sizes: nx, ny in [32,128] (multiples
    of 4), nz in [32,200], dx 2-8 um, V 50-400 V, LET log-uniform 1-1000
    keV/um, b 5-20 um, 1-500 tracks.  Draws per simulation: 8 uniforms."""
    u = uniform01(seed, 8 * n).reshape(n, 8)
    out = []
    for k in range(n):
        nx = 32 + 4 * int(u[k, 0] * 25)
        ny = 32 + 4 * int(u[k, 1] * 25)
        nz = 32 + int(u[k, 2] * 169)
        dx = (2.0 + 6.0 * u[k, 3]) * 1e-4
        V = 50.0 + 350.0 * u[k, 4]
        let = 10.0 ** (3.0 * u[k, 5])
        b = (5.0 + 15.0 * u[k, 6]) * 1e-4
        nt = 1 + int(u[k, 7] * 500)
        out.append(dict(nx=nx, ny=ny, nz=nz, dx_cm=dx, voltage_V=V, let=let, b_cm=b,
                        n_tracks=nt, seed=seed * 1000 + k))
    return out


def batch_tracks(desc) -> TrackList:
    """Tracks of one batched simulation: uniform (x, y), one LET, one b."""
    return uniform_tracks(desc["seed"], desc["n_tracks"], desc["nx"] * desc["dx_cm"],
                          desc["ny"] * desc["dx_cm"], desc["b_cm"], let=desc["let"])


# ---------------------------------------------------------------------------
# surrogate workload: configurations described by six inputs
# ---------------------------------------------------------------------------

SURROGATE_DX_CM = 5e-4           # one grid spacing for every surrogate configuration
SURROGATE_NX = 48                # lateral section 48 x 48 cells = 0.24 mm x 0.24 mm
SURROGATE_SECTION_CM = SURROGATE_NX * SURROGATE_DX_CM
SURROGATE_CHECK = 64             # pulse periods are whole multiples of this many steps


def surrogate_configs(seed: int, n: int):
    """n seeded configurations for the surrogate.

    Inputs (the six the network sees): LET (log-uniform 1-1000 keV/um),
    voltage (50-400 V), gap (20-100 cells of 5 um: 0.1-0.5 mm), b (5-20 um),
    tracks per pulse (1-500 on the fixed 0.24 mm section) and pulse period
    (0 = a single pulse with probability 1/2, else log-uniform 1-30 us for a
    train of 4 pulses).  The grid is the same for every configuration (dx =
    5 um, 48 x 48 cells) and the gap is a whole number of cells, so every
    input is represented exactly and f is a continuous function of them: a
    grid spacing that follows b would round the section and the gap to whole
    cells differently for nearby inputs, and the simulated track density
    would jump with it.  Draws per configuration: 8 uniforms.
    """
    u = uniform01(seed, 8 * n).reshape(n, 8)
    out = []
    dx, nx = SURROGATE_DX_CM, SURROGATE_NX
    for k in range(n):
        let = 10.0 ** (3.0 * u[k, 0])
        V = 50.0 + 350.0 * u[k, 1]
        nz = 20 + int(u[k, 2] * 81)
        b = (5.0 + 15.0 * u[k, 3]) * 1e-4
        ntr = 1 + int(u[k, 4] * 500)
        period = 0.0 if u[k, 5] < 0.5 else 10.0 ** (-6.0 + 1.5 * u[k, 6])
        out.append(dict(let=let, voltage_V=V, b_cm=b, n_tracks=ntr, period_s=period,
                        pulses=1 if period == 0.0 else 4, nx=nx, ny=nx, nz=nz, dx_cm=dx,
                        gap_cm=nz * dx, seed=seed * 100003 + k))
    return out


# Roberts' R2 low-discrepancy sequence (generalised golden ratio g, the real
# root of g^3 = g + 1): point i = frac(0.5 + i (1/g, 1/g^2)).
_R2_G = 1.32471795724474602596


def r2_points(n: int) -> np.ndarray:
    """First n points of the R2 sequence in [0,1)^2 ([n][2])."""
    i = np.arange(1, n + 1, dtype=np.float64)
    a = np.array([1.0 / _R2_G, 1.0 / _R2_G ** 2])
    return np.mod(0.5 + i[:, None] * a[None, :], 1.0)


def surrogate_tracks(cfg) -> TrackList:
    """Tracks of one pulse of a surrogate configuration: uniformly spread
    over the section on the R2 sequence, so that f is a function of the six
    inputs (random positions make f scatter by up to ~1e-2 between draws)."""
    L = cfg["nx"] * cfg["dx_cm"]
    p = r2_points(cfg["n_tracks"]) * L
    n = cfg["n_tracks"]
    return TrackList(p[:, 0].copy(), p[:, 1].copy(), np.full(n, float(cfg["let"])), np.full(n, float(cfg["b_cm"])))


def surrogate_features(cfg, period_s=None) -> np.ndarray:
    """The six network inputs, each on a log scale: log10 of LET (keV/um),
    voltage (V), gap (cm), b (cm), tracks per pulse, and pulse period + 1 us
    (s; the period actually simulated when given, 0 for a single pulse)."""
    p = cfg["period_s"] if period_s is None else period_s
    return np.log10(np.array([cfg["let"], cfg["voltage_V"], cfg["gap_cm"], cfg["b_cm"],
                              float(cfg["n_tracks"]), p + 1e-6], dtype=np.float64))


def mlp_init(seed: int, members: int = 5) -> np.ndarray:
    """Initial surrogate weights, [members][n_params] float64: every weight
    uniform in [-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64, biases 0.
    Layout per member: W1 [256][6], b1, W2 [256][256], b2, W3, b3, W4, b4,
    W5 [1][256], b5."""
    shapes = [(256, 6), (256,), (256, 256), (256,), (256, 256), (256,), (256, 256), (256,), (1, 256), (1,)]
    n = int(sum(np.prod(s) for s in shapes))
    out = np.zeros((members, n))
    for m in range(members):
        o = 0
        for q, s in enumerate(shapes):
            k = int(np.prod(s))
            if len(s) == 2:
                u = uniform01(seed * 7 + 1000 * m + q, k)
                out[m, o:o + k] = (2.0 * u - 1.0) / math.sqrt(s[1])
            o += k
    return out
