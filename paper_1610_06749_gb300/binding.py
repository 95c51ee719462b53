"""ctypes binding of ``libiontracks.so`` (include/iontracks.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the C names (``it_create``, ``it_step``, ...)
and raise ``ItError`` on a non-zero return code.  ``Simulation`` bundles a
context with numpy/torch conveniences.  There is no CPU fallback: if the
shared library is missing this module raises on import of the library.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiontracks.so")

IT_OK, IT_EINVAL, IT_ENOMEM, IT_ECUDA, IT_EUNSTABLE, IT_ETIMEOUT, IT_ESTATE = 0, -1, -2, -3, -4, -5, -6
IT_FP32, IT_FP64 = 0, 1
IT_PERIODIC, IT_ABSORBING = 0, 1
IT_LAX_WENDROFF, IT_UPWIND = 0, 1
IT_KERNEL_AUTO, IT_KERNEL_SIMPLE, IT_KERNEL_ZMARCH, IT_KERNEL_ZMARCH2 = 0, 1, 2, 3

_ERRNAMES = {IT_EINVAL: "IT_EINVAL", IT_ENOMEM: "IT_ENOMEM", IT_ECUDA: "IT_ECUDA",
             IT_EUNSTABLE: "IT_EUNSTABLE", IT_ETIMEOUT: "IT_ETIMEOUT", IT_ESTATE: "IT_ESTATE"}


class ItError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class it_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class it_params(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double * 2), ("D", ctypes.c_double * 2), ("alpha", ctypes.c_double),
                ("W_eV", ctypes.c_double), ("gap_cm", ctypes.c_double), ("voltage_V", ctypes.c_double),
                ("precision", ctypes.c_int32), ("lateral_bc", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("cfl_safety", ctypes.c_double), ("react_kappa", ctypes.c_double),
                ("n_peak_cm3", ctypes.c_double), ("space_charge", ctypes.c_int32), ("dt_ladder", ctypes.c_int32)]


class it_tallies_t(ctypes.Structure):
    _fields_ = [("released", ctypes.c_double * 2), ("collected_anode", ctypes.c_double * 2),
                ("collected_cathode", ctypes.c_double * 2), ("lost_lateral", ctypes.c_double * 2),
                ("in_domain", ctypes.c_double * 2), ("recombined", ctypes.c_double), ("f", ctypes.c_double),
                ("t_s", ctypes.c_double), ("dt_s", ctypes.c_double), ("steps", ctypes.c_int64),
                ("n_min", ctypes.c_double * 2), ("n_max", ctypes.c_double * 2),
                ("space_charge", ctypes.c_double * 2)]


class it_sim_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx_cm", ctypes.c_double), ("dt_s", ctypes.c_double), ("voltage_V", ctypes.c_double),
                ("n_peak_cm3", ctypes.c_double)]


class it_steady_t(ctypes.Structure):
    _fields_ = [("f_ss", ctypes.c_double), ("f_ss_stderr", ctypes.c_double), ("f_window", ctypes.c_double),
                ("departed", ctypes.c_double), ("released", ctypes.c_double), ("windows", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("stop", ctypes.c_int32), ("pad_", ctypes.c_int32)]


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, I64, SZ = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        DP = ctypes.POINTER(ctypes.c_double)
        I64P = ctypes.POINTER(ctypes.c_int64)
        IP = ctypes.POINTER(ctypes.c_int)
        sig = {
            "it_version": (ctypes.c_char_p, []),
            "it_last_error": (ctypes.c_char_p, []),
            "it_params_default": (I, [ctypes.POINTER(it_params)]),
            "it_auto_dt": (I, [ctypes.POINTER(it_params), D, DP]),
            "it_ladder_dt": (I, [ctypes.POINTER(it_params), D, D, D, DP]),
            "it_peak_density": (I, [I64, DP, DP, D, DP]),
            "it_state_bytes": (I, [it_grid, ctypes.c_int32, ctypes.POINTER(SZ)]),
            "it_create": (I, [it_grid, D, D, ctypes.POINTER(it_params), ctypes.POINTER(P)]),
            "it_create_ex": (I, [it_grid, D, D, ctypes.POINTER(it_params), P, SZ, P, ctypes.POINTER(P)]),
            "it_deposit_tracks": (I, [P, I64, DP, DP, DP]),
            "it_deposit_tracks_device": (I, [P, I64, P]),
            "it_deposit_tracks_angled": (I, [P, I64, DP, DP, DP, DP]),
            "it_schedule_tracks": (I, [P, I64, DP, DP, DP, I64P]),
            "it_step": (I, [P, I64]),
            "it_run_to_completion": (I, [P, D, I64, I64, I64P]),
            "it_run_to_steady_state": (I, [P, I64, D, I64, ctypes.POINTER(it_steady_t)]),
            "it_tallies": (I, [P, ctypes.POINTER(it_tallies_t)]),
            "it_get_density": (I, [P, I, P, SZ]),
            "it_set_density": (I, [P, P, P, SZ]),
            "it_reset": (I, [P]),
            "it_retime": (I, [P, D]),
            "it_dt_log": (I, [P, I64, I64P, DP, DP, I64P]),
            "it_batch_retime": (I, [P]),
            "it_device_state": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]),
            "it_set_launch": (I, [P, I, I, I, I]),
            "it_set_launch_ex": (I, [P, I, I, I, I, I]),
            "it_autotune": (I, [P, I, I, DP]),
            "it_get_launch": (I, [P, IP, IP, IP, IP, IP]),
            "it_step_noalloc": (I, [it_grid, D, D, ctypes.POINTER(it_params), P, P, P, P, P, P]),
            "it_set_wait_limit": (I, [P, I64]),
            "it_test_withhold_load": (I, [P, I]),
            "it_batch_create": (I, [ctypes.c_int32, ctypes.POINTER(it_sim_desc), ctypes.POINTER(it_params),
                                    ctypes.POINTER(P)]),
            "it_batch_deposit_tracks": (I, [P, ctypes.c_int32, I64, DP, DP, DP]),
            "it_batch_set_chunk": (I, [P, I64]),
            "it_batch_autotune": (I, [P, ctypes.c_int32, ctypes.POINTER(D)]),
            "it_batch_set_pulses": (I, [P, ctypes.c_int32, ctypes.c_int32, I64]),
            "it_batch_run": (I, [P, D, I64, I64, I64P]),
            "it_batch_tallies": (I, [P, ctypes.c_int32, ctypes.POINTER(it_tallies_t)]),
            "it_batch_get_density": (I, [P, ctypes.c_int32, I, P, SZ]),
            "it_batch_destroy": (I, [P]),
            "it_mlp_create": (I, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(P)]),
            "it_mlp_set_params": (I, [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), I64]),
            "it_mlp_get_params": (I, [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), I64]),
            "it_mlp_set_normalization": (I, [P, DP, DP]),
            "it_mlp_fit_normalization": (I, [P, I64, DP]),
            "it_mlp_set_data": (I, [P, I64, DP, DP]),
            "it_mlp_train": (I, [P, ctypes.c_int32, ctypes.c_int32, D, ctypes.c_uint64, DP]),
            "it_mlp_loss_grad": (I, [P, I64, DP, DP, ctypes.POINTER(ctypes.c_float), DP]),
            "it_mlp_adam_step": (I, [P, D]),
            "it_mlp_predict": (I, [P, I64, DP, DP, DP, DP]),
            "it_mlp_destroy": (I, [P]),
            "it_destroy": (I, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != IT_OK:
        raise ItError(rc, lib().it_last_error().decode(errors="replace"))
    return rc


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# thin wrappers with the C names
# --------------------------------------------------------------------------

def it_version() -> str:
    return lib().it_version().decode()


def it_last_error() -> str:
    return lib().it_last_error().decode(errors="replace")


def it_params_default(**kw) -> it_params:
    p = it_params()
    _check(lib().it_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k in ("mu", "D"):
            getattr(p, k)[0], getattr(p, k)[1] = float(v[0]), float(v[1])
        else:
            setattr(p, k, v)
    return p


def it_ladder_dt(p: it_params, dx_cm: float, dt_s: float, n_max: float) -> float:
    out = ctypes.c_double()
    _check(lib().it_ladder_dt(ctypes.byref(p), float(dx_cm), float(dt_s), float(n_max), ctypes.byref(out)))
    return out.value


def it_auto_dt(p: it_params, dx_cm: float) -> float:
    out = ctypes.c_double()
    _check(lib().it_auto_dt(ctypes.byref(p), float(dx_cm), ctypes.byref(out)))
    return out.value


def it_peak_density(let_keV_um, b_cm, W_eV=34.0) -> float:
    L, b = _f64(let_keV_um), _f64(b_cm)
    out = ctypes.c_double()
    _check(lib().it_peak_density(L.size, _dp(L), _dp(b), float(W_eV), ctypes.byref(out)))
    return out.value


def it_state_bytes(nx, ny, nz, precision=IT_FP32) -> int:
    out = ctypes.c_size_t()
    _check(lib().it_state_bytes(it_grid(nx, ny, nz), precision, ctypes.byref(out)))
    return out.value


def it_create(nx, ny, nz, dx_cm, dt_s, p: it_params):
    h = ctypes.c_void_p()
    _check(lib().it_create(it_grid(nx, ny, nz), float(dx_cm), float(dt_s), ctypes.byref(p), ctypes.byref(h)))
    return h


def it_create_ex(nx, ny, nz, dx_cm, dt_s, p: it_params, dev_state: int, nbytes: int, stream: int):
    h = ctypes.c_void_p()
    _check(lib().it_create_ex(it_grid(nx, ny, nz), float(dx_cm), float(dt_s), ctypes.byref(p),
                              ctypes.c_void_p(dev_state), nbytes, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def it_deposit_tracks(h, xy_cm, let_keV_um, b_cm):
    xy, L, b = _f64(xy_cm).reshape(-1), _f64(let_keV_um), _f64(b_cm)
    _check(lib().it_deposit_tracks(h, L.size, _dp(xy), _dp(L), _dp(b)))


def it_deposit_tracks_angled(h, xy_cm, let_keV_um, b_cm, theta_rad):
    xy, L, b, th = _f64(xy_cm).reshape(-1), _f64(let_keV_um), _f64(b_cm), _f64(theta_rad)
    if not (th.size == L.size == b.size and xy.size == 2 * L.size):
        raise ValueError("track arrays differ in length")
    _check(lib().it_deposit_tracks_angled(h, L.size, _dp(xy), _dp(L), _dp(b), _dp(th)))


def it_deposit_tracks_device(h, n: int, dev_tracks: int):
    """dev_tracks: device address of n x 4 doubles (x, y, LET, b)."""
    _check(lib().it_deposit_tracks_device(h, int(n), ctypes.c_void_p(dev_tracks)))


def it_schedule_tracks(h, xy_cm, let_keV_um, b_cm, step_idx):
    xy, L, b = _f64(xy_cm).reshape(-1), _f64(let_keV_um), _f64(b_cm)
    s = np.ascontiguousarray(step_idx, dtype=np.int64)
    _check(lib().it_schedule_tracks(h, L.size, _dp(xy), _dp(L), _dp(b),
                                    s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))


def it_step(h, n_steps: int):
    _check(lib().it_step(h, int(n_steps)))


def it_run_to_completion(h, tol=1e-6, max_steps=10_000_000, check_every=64) -> int:
    done = ctypes.c_int64()
    _check(lib().it_run_to_completion(h, float(tol), int(max_steps), int(check_every), ctypes.byref(done)))
    return done.value


def it_run_to_steady_state(h, window_steps=1000, tol=1e-5, max_steps=10_000_000) -> dict:
    """Returns the it_steady_t fields as a dict (f_ss, f_ss_stderr, f_window,
    departed, released, windows, steps, stop: 0 steady / 1 step limit)."""
    out = it_steady_t()
    _check(lib().it_run_to_steady_state(h, int(window_steps), float(tol), int(max_steps), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in it_steady_t._fields_ if k != "pad_"}


def it_tallies(h) -> it_tallies_t:
    t = it_tallies_t()
    _check(lib().it_tallies(h, ctypes.byref(t)))
    return t


def it_get_density(h, species: int, out: np.ndarray):
    _check(lib().it_get_density(h, int(species), out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
    return out


def it_set_density(h, plus: np.ndarray, minus: np.ndarray):
    _check(lib().it_set_density(h, plus.ctypes.data_as(ctypes.c_void_p), minus.ctypes.data_as(ctypes.c_void_p),
                                plus.nbytes))


def it_retime(h, dt_s=0.0):
    _check(lib().it_retime(h, float(dt_s)))


def it_batch_retime(h):
    _check(lib().it_batch_retime(h))


def it_reset(h):
    _check(lib().it_reset(h))


def it_dt_log(h):
    """The time-step log: a list of (first step, dt, deciding n_max)."""
    n = ctypes.c_int64()
    _check(lib().it_dt_log(h, 0, None, None, None, ctypes.byref(n)))
    m = n.value
    st = (ctypes.c_int64 * m)()
    dt = (ctypes.c_double * m)()
    nm = (ctypes.c_double * m)()
    _check(lib().it_dt_log(h, m, st, dt, nm, ctypes.byref(n)))
    return [(int(st[q]), float(dt[q]), float(nm[q])) for q in range(m)]


def it_device_state(h):
    p, m, s = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().it_device_state(h, ctypes.byref(p), ctypes.byref(m), ctypes.byref(s)))
    return p.value, m.value, s.value


def it_set_launch(h, kernel=IT_KERNEL_AUTO, tile_rows=0, ctas_per_sm=0, stages=0):
    _check(lib().it_set_launch(h, int(kernel), int(tile_rows), int(ctas_per_sm), int(stages)))


def it_set_launch_ex(h, kernel=IT_KERNEL_AUTO, tile_rows=0, ctas_per_sm=0, stages=0, grid=0):
    _check(lib().it_set_launch_ex(h, int(kernel), int(tile_rows), int(ctas_per_sm), int(stages), int(grid)))


def it_autotune(h, trial_steps=8, flags=0) -> float:
    us = ctypes.c_double()
    _check(lib().it_autotune(h, int(trial_steps), int(flags), ctypes.byref(us)))
    return us.value


def it_get_launch(h):
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().it_get_launch(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(("kernel", "tile_rows", "ctas_per_sm", "stages", "ctas"), [x.value for x in v]))


def it_step_noalloc(nx, ny, nz, dx_cm, dt_s, p: it_params, dev_plus: int, dev_minus: int,
                    dev_out_plus: int, dev_out_minus: int, dev_tallies7: int, stream: int = 0):
    """One step on caller-owned device buffers; allocates nothing (device
    addresses as ints, e.g. torch tensors' data_ptr())."""
    _check(lib().it_step_noalloc(it_grid(nx, ny, nz), float(dx_cm), float(dt_s), ctypes.byref(p),
                                 ctypes.c_void_p(dev_plus), ctypes.c_void_p(dev_minus),
                                 ctypes.c_void_p(dev_out_plus), ctypes.c_void_p(dev_out_minus),
                                 ctypes.c_void_p(dev_tallies7), ctypes.c_void_p(stream)))


def it_set_wait_limit(h, cycles: int):
    _check(lib().it_set_wait_limit(h, int(cycles)))


def it_test_withhold_load(h, on: bool):
    _check(lib().it_test_withhold_load(h, 1 if on else 0))


def it_destroy(h):
    if h:
        _check(lib().it_destroy(h))


def it_batch_create(descs, p: it_params):
    arr = (it_sim_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().it_batch_create(len(descs), arr, ctypes.byref(p), ctypes.byref(h)))
    return h


def it_batch_deposit_tracks(h, sim, xy_cm, let_keV_um, b_cm):
    xy, L, b = _f64(xy_cm).reshape(-1), _f64(let_keV_um), _f64(b_cm)
    _check(lib().it_batch_deposit_tracks(h, int(sim), L.size, _dp(xy), _dp(L), _dp(b)))


def it_batch_set_pulses(h, sim, count, period_steps):
    _check(lib().it_batch_set_pulses(h, int(sim), int(count), int(period_steps)))


def it_batch_set_chunk(h, cells_per_block):
    _check(lib().it_batch_set_chunk(h, int(cells_per_block)))


def it_batch_autotune(h, trial_steps=8) -> float:
    us = ctypes.c_double()
    _check(lib().it_batch_autotune(h, int(trial_steps), ctypes.byref(us)))
    return us.value


def it_batch_run(h, tol=1e-6, max_steps=10_000_000, check_every=64) -> int:
    n = ctypes.c_int64()
    _check(lib().it_batch_run(h, float(tol), int(max_steps), int(check_every), ctypes.byref(n)))
    return n.value


def it_batch_tallies(h, sim) -> it_tallies_t:
    t = it_tallies_t()
    _check(lib().it_batch_tallies(h, int(sim), ctypes.byref(t)))
    return t


def it_batch_get_density(h, sim, species, out: np.ndarray):
    _check(lib().it_batch_get_density(h, int(sim), int(species), out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
    return out


def it_batch_destroy(h):
    if h:
        _check(lib().it_batch_destroy(h))


IT_MLP_INPUTS, IT_MLP_HIDDEN, IT_MLP_PARAMS = 6, 256, 199425


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def it_mlp_create(members=5, max_batch=1024):
    h = ctypes.c_void_p()
    _check(lib().it_mlp_create(int(members), int(max_batch), ctypes.byref(h)))
    return h


def it_mlp_set_params(h, member, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().it_mlp_set_params(h, int(member), _fp(a), a.size))


def it_mlp_get_params(h, member):
    out = np.empty(IT_MLP_PARAMS, dtype=np.float32)
    _check(lib().it_mlp_get_params(h, int(member), _fp(out), out.size))
    return out


def it_mlp_set_normalization(h, mean6, std6):
    m, s = _f64(mean6), _f64(std6)
    _check(lib().it_mlp_set_normalization(h, _dp(m), _dp(s)))


def it_mlp_fit_normalization(h, x):
    a = _f64(x).reshape(-1, IT_MLP_INPUTS)
    _check(lib().it_mlp_fit_normalization(h, a.shape[0], _dp(a)))


def it_mlp_set_data(h, x, y):
    a, b = _f64(x).reshape(-1, IT_MLP_INPUTS), _f64(y)
    _check(lib().it_mlp_set_data(h, a.shape[0], _dp(a), _dp(b)))


def it_mlp_train(h, epochs, batch, lr, seed):
    loss = np.zeros(max(int(epochs), 1))
    _check(lib().it_mlp_train(h, int(epochs), int(batch), float(lr), ctypes.c_uint64(seed & (2 ** 64 - 1)), _dp(loss)))
    return loss[:int(epochs)]


def it_mlp_loss_grad(h, members, x, y):
    a, b = _f64(x).reshape(-1, IT_MLP_INPUTS), _f64(y)
    g = np.empty((members, IT_MLP_PARAMS), dtype=np.float32)
    loss = np.empty(members)
    _check(lib().it_mlp_loss_grad(h, a.shape[0], _dp(a), _dp(b), _fp(g), _dp(loss)))
    return loss, g


def it_mlp_adam_step(h, lr):
    _check(lib().it_mlp_adam_step(h, float(lr)))


def it_mlp_predict(h, members, x):
    a = _f64(x).reshape(-1, IT_MLP_INPUTS)
    n = a.shape[0]
    mean, spread, per = np.empty(n), np.empty(n), np.empty((n, members))
    _check(lib().it_mlp_predict(h, n, _dp(a), _dp(mean), _dp(spread), _dp(per)))
    return mean, spread, per


def it_mlp_destroy(h):
    if h:
        _check(lib().it_mlp_destroy(h))


# --------------------------------------------------------------------------
# convenience wrapper
# --------------------------------------------------------------------------

@dataclass
class Tallies:
    released: np.ndarray
    collected_anode: np.ndarray
    collected_cathode: np.ndarray
    lost_lateral: np.ndarray
    in_domain: np.ndarray
    recombined: float
    f: float
    t_s: float
    dt_s: float
    steps: int
    n_min: np.ndarray
    n_max: np.ndarray
    space_charge: np.ndarray   # ions added per species by the space-charge term (0 when off)

    @property
    def collected(self):
        return self.collected_anode + self.collected_cathode

    @classmethod
    def from_c(cls, t: it_tallies_t):
        a = lambda x: np.array([x[0], x[1]])
        return cls(a(t.released), a(t.collected_anode), a(t.collected_cathode), a(t.lost_lateral),
                   a(t.in_domain), t.recombined, t.f, t.t_s, t.dt_s, t.steps, a(t.n_min), a(t.n_max),
                   a(t.space_charge))


class Batch:
    """Many simulations advanced together (see it_batch_create)."""

    def __init__(self, descs, mu=(1.73, 1.87), D=(0.037, 0.037), alpha=1.6e-6, W_eV=34.0,
                 lateral_bc=IT_PERIODIC, scheme=IT_LAX_WENDROFF, cfl_safety=1.0, react_kappa=0.5,
                 space_charge=False, dt_ladder=False):
        self.descs = [it_sim_desc(int(d["nx"]), int(d["ny"]), int(d["nz"]), float(d["dx_cm"]),
                                  float(d.get("dt_s", 0.0)), float(d["voltage_V"]), float(d.get("n_peak_cm3", 0.0)))
                      for d in descs]
        p = it_params_default(mu=mu, D=D, alpha=alpha, W_eV=W_eV, lateral_bc=lateral_bc, scheme=scheme,
                              cfl_safety=cfl_safety, react_kappa=react_kappa, gap_cm=1.0,
                              space_charge=int(bool(space_charge)), dt_ladder=int(bool(dt_ladder)))
        self.h = it_batch_create(self.descs, p)

    def deposit(self, sim, x_cm, y_cm, let_keV_um, b_cm):
        xy = np.stack([np.asarray(x_cm, np.float64), np.asarray(y_cm, np.float64)], axis=1)
        it_batch_deposit_tracks(self.h, sim, xy, let_keV_um, b_cm)

    def set_pulses(self, sim, count, period_steps):
        it_batch_set_pulses(self.h, sim, count, period_steps)

    def retime(self):
        """dt of every automatic-dt simulation from its deposited peak density."""
        it_batch_retime(self.h)

    def set_chunk(self, cells):
        it_batch_set_chunk(self.h, cells)

    def autotune(self, trial_steps=8) -> float:
        return it_batch_autotune(self.h, trial_steps)

    def run(self, tol=1e-6, max_steps=10_000_000, check_every=64):
        return it_batch_run(self.h, tol, max_steps, check_every)

    def tallies(self, sim) -> "Tallies":
        return Tallies.from_c(it_batch_tallies(self.h, sim))

    def density(self, sim, species):
        d = self.descs[sim]
        out = np.empty((d.nz, d.ny, d.nx), dtype=np.float32)
        return it_batch_get_density(self.h, sim, species, out)

    def close(self):
        if getattr(self, "h", None):
            it_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Simulation:
    """One simulation context on the current CUDA device.

    ``torch_state=True`` allocates the density state as a torch tensor and
    runs on torch's current stream (``it_create_ex``); otherwise the library
    owns its memory and stream.
    """

    def __init__(self, nx, ny, nz, dx_cm, voltage_V, dt_s=0.0, mu=(1.73, 1.87), D=(0.037, 0.037),
                 alpha=1.6e-6, W_eV=34.0, precision=IT_FP32, lateral_bc=IT_PERIODIC,
                 scheme=IT_LAX_WENDROFF, kernel=IT_KERNEL_AUTO, n_peak_cm3=0.0, cfl_safety=1.0,
                 react_kappa=0.5, torch_state=False, space_charge=False, dt_ladder=False):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.precision = precision
        self.p = it_params_default(mu=mu, D=D, alpha=alpha, W_eV=W_eV, gap_cm=self.nz * dx_cm,
                                   voltage_V=voltage_V, precision=precision, lateral_bc=lateral_bc,
                                   scheme=scheme, kernel=kernel, n_peak_cm3=n_peak_cm3,
                                   cfl_safety=cfl_safety, react_kappa=react_kappa,
                                   space_charge=int(bool(space_charge)), dt_ladder=int(bool(dt_ladder)))
        self._state = None
        if torch_state:
            import torch
            nbytes = it_state_bytes(nx, ny, nz, precision)
            self._state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            self.h = it_create_ex(nx, ny, nz, dx_cm, dt_s, self.p, self._state.data_ptr(), nbytes, stream)
        else:
            self.h = it_create(nx, ny, nz, dx_cm, dt_s, self.p)

    @property
    def dtype(self):
        return np.float64 if self.precision == IT_FP64 else np.float32

    def deposit(self, x_cm, y_cm, let_keV_um, b_cm):
        xy = np.stack([np.asarray(x_cm, np.float64), np.asarray(y_cm, np.float64)], axis=1)
        it_deposit_tracks(self.h, xy, let_keV_um, b_cm)

    def deposit_angled(self, x_cm, y_cm, let_keV_um, b_cm, theta_rad):
        """Tracks at angle theta in [0, pi/2] to the field, axes through
        (x, y, d/2), rotated in the x-z plane (it_deposit_tracks_angled)."""
        xy = np.stack([np.atleast_1d(np.asarray(x_cm, np.float64)), np.atleast_1d(np.asarray(y_cm, np.float64))],
                      axis=1)
        it_deposit_tracks_angled(self.h, xy, np.atleast_1d(let_keV_um), np.atleast_1d(b_cm),
                                 np.atleast_1d(theta_rad))

    def schedule(self, x_cm, y_cm, let_keV_um, b_cm, step_idx):
        xy = np.stack([np.asarray(x_cm, np.float64), np.asarray(y_cm, np.float64)], axis=1)
        it_schedule_tracks(self.h, xy, let_keV_um, b_cm, step_idx)

    def step(self, n=1):
        it_step(self.h, n)

    def run_to_completion(self, tol=1e-6, max_steps=10_000_000, check_every=64):
        return it_run_to_completion(self.h, tol, max_steps, check_every)

    def run_to_steady_state(self, window_steps=1000, tol=1e-5, max_steps=10_000_000):
        return it_run_to_steady_state(self.h, window_steps, tol, max_steps)

    def tallies(self) -> Tallies:
        return Tallies.from_c(it_tallies(self.h))

    def density(self, species) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx), dtype=self.dtype)
        return it_get_density(self.h, species, out)

    def set_density(self, plus, minus):
        shape = (self.nz, self.ny, self.nx)
        p = np.ascontiguousarray(np.broadcast_to(plus, shape), dtype=self.dtype)
        m = np.ascontiguousarray(np.broadcast_to(minus, shape), dtype=self.dtype)
        it_set_density(self.h, p, m)

    def reset(self):
        it_reset(self.h)

    def retime(self, dt_s=0.0):
        """Before the first step: dt_s > 0 sets it; 0 derives it from the
        largest density of the current (deposited) state."""
        it_retime(self.h, dt_s)

    def dt_log(self):
        """[(first step, dt, deciding n_max)] of every time step used."""
        return it_dt_log(self.h)

    def launch(self):
        return it_get_launch(self.h)

    def set_launch(self, kernel=IT_KERNEL_AUTO, tile_rows=0, ctas_per_sm=0, stages=0, grid=0):
        it_set_launch_ex(self.h, kernel, tile_rows, ctas_per_sm, stages, grid)

    def autotune(self, trial_steps=8, force=False) -> float:
        """Pick the fastest step-kernel launch shape on the current state
        (which is left unchanged); returns its time per step in us (-1 if
        the shape came from the per-process cache)."""
        return it_autotune(self.h, trial_steps, 1 if force else 0)

    def close(self):
        if getattr(self, "h", None):
            it_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
