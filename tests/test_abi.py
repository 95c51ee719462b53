"""The C-ABI library builds, loads and exports what include/iontracks.h
declares; host-only entry points work without a GPU and agree with the
oracle's time-step rule; device entry points fail loudly without a GPU."""
import ctypes
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle.oracle as o
from paper_1610_06749_gb300 import build as libbuild
from paper_1610_06749_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iontracks.h")


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return B.lib()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(it_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ["it_create", "it_create_ex", "it_deposit_tracks", "it_schedule_tracks", "it_step",
                 "it_tallies", "it_destroy", "it_run_to_completion", "it_get_density", "it_set_density",
                 "it_auto_dt", "it_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(L):
    for n in declared_symbols():
        assert hasattr(B, n), n


def test_version_and_defaults(L):
    assert "sm_103a" in B.it_version()
    p = B.it_params_default()
    assert tuple(p.mu) == (1.73, 1.87) and tuple(p.D) == (0.037, 0.037)
    assert p.alpha == 1.6e-6 and p.W_eV == 34.0 and p.react_kappa == 0.5


@pytest.mark.parametrize("scheme", [B.IT_LAX_WENDROFF, B.IT_UPWIND])
@pytest.mark.parametrize("dx,V,d", [(2e-4, 200.0, 0.02), (5e-4, 50.0, 0.2), (8e-4, 300.0, 0.2048)])
def test_auto_dt_matches_oracle_rule(L, scheme, dx, V, d):
    npk = o.peak_track_density([1000.0], [1e-3])
    for n_peak in (0.0, npk):
        p = B.it_params_default(gap_cm=d, voltage_V=V, scheme=scheme, n_peak_cm3=n_peak)
        got = B.it_auto_dt(p, dx)
        want = o.dt_rule(dx, V, d, (1.73, 1.87), (0.037, 0.037), 1.6e-6, n_peak=n_peak,
                         scheme=o.SCHEME_UPWIND if scheme == B.IT_UPWIND else o.SCHEME_LAX_WENDROFF)
        assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("n_peak", [1e12, 1e13, 9.4e13])
def test_auto_dt_with_space_charge_matches_oracle_rule(L, n_peak):
    """With the space-charge term on, the automatic dt also keeps
    max mu q/eps0 n_peak dt <= kappa, exactly as the oracle's rule."""
    for dx, V, d in [(5e-4, 200.0, 0.2), (2e-4, 50.0, 0.02)]:
        p = B.it_params_default(gap_cm=d, voltage_V=V, n_peak_cm3=n_peak, space_charge=1)
        want = o.dt_rule(dx, V, d, (1.73, 1.87), (0.037, 0.037), 1.6e-6, n_peak=n_peak, space_charge=True)
        assert B.it_auto_dt(p, dx) == pytest.approx(want, rel=1e-14)
        off = B.it_auto_dt(B.it_params_default(gap_cm=d, voltage_V=V, n_peak_cm3=n_peak), dx)
        assert B.it_auto_dt(p, dx) <= off


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "iontracks.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
#define S(T) printf(#T " sizeof %zu\n", sizeof(T));
int main(void) {
    S(it_params) F(it_params, mu) F(it_params, D) F(it_params, alpha) F(it_params, W_eV)
    F(it_params, gap_cm) F(it_params, voltage_V) F(it_params, precision) F(it_params, lateral_bc)
    F(it_params, scheme) F(it_params, kernel) F(it_params, cfl_safety) F(it_params, react_kappa)
    F(it_params, n_peak_cm3) F(it_params, space_charge) F(it_params, dt_ladder)
    S(it_tallies_t) F(it_tallies_t, released) F(it_tallies_t, collected_anode)
    F(it_tallies_t, collected_cathode) F(it_tallies_t, lost_lateral) F(it_tallies_t, in_domain)
    F(it_tallies_t, recombined) F(it_tallies_t, f) F(it_tallies_t, t_s) F(it_tallies_t, dt_s)
    F(it_tallies_t, steps) F(it_tallies_t, n_min) F(it_tallies_t, n_max) F(it_tallies_t, space_charge)
    S(it_sim_desc) F(it_sim_desc, nx) F(it_sim_desc, ny) F(it_sim_desc, nz) F(it_sim_desc, dx_cm)
    F(it_sim_desc, dt_s) F(it_sim_desc, voltage_V) F(it_sim_desc, n_peak_cm3)
    S(it_grid)
    S(it_steady_t) F(it_steady_t, f_ss) F(it_steady_t, f_ss_stderr) F(it_steady_t, f_window)
    F(it_steady_t, departed) F(it_steady_t, released) F(it_steady_t, windows) F(it_steady_t, steps)
    F(it_steady_t, stop)
    return 0;
}
"""


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes struct has the size and field offsets the C compiler
    gives the header's struct."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        tname, field, val = line.split()
        cls = getattr(B, tname)
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(val), (tname, field, got, val)
        seen += 1
    assert seen == 48


def test_peak_density_and_state_bytes(L):
    let, b = np.array([1.0, 1000.0, 10.0]), np.array([1e-3, 1e-3, 5e-4])
    assert B.it_peak_density(let, b) == pytest.approx(o.peak_track_density(let, b), rel=1e-15)
    n = B.it_state_bytes(256, 256, 400, B.IT_FP32)
    assert n == 4 * 256 * 256 * 400 * 4
    assert B.it_state_bytes(48, 48, 100, B.IT_FP64) == 4 * ((48 * 48 * 100 * 8 + 255) // 256 * 256)


def test_invalid_parameters_are_rejected(L):
    p = B.it_params_default(gap_cm=0.02, voltage_V=200.0)
    with pytest.raises(B.ItError) as e:
        B.it_auto_dt(p, -1.0)
    assert e.value.code == B.IT_EINVAL
    p2 = B.it_params_default(gap_cm=0.021, voltage_V=200.0)      # gap != nz * dx
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, 0.0, p2)
    assert e.value.code == B.IT_EINVAL
    p3 = B.it_params_default(gap_cm=0.02, voltage_V=float("nan"))
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, 0.0, p3)
    assert e.value.code == B.IT_EINVAL
    p4 = B.it_params_default(gap_cm=0.02, voltage_V=200.0, space_charge=2)
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, 0.0, p4)
    assert e.value.code == B.IT_EINVAL
    # dt above the von Neumann bound
    dt = B.it_auto_dt(p, 2e-4)
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, dt * 1.01, p)
    assert e.value.code == B.IT_EINVAL


def test_create_without_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = B.it_params_default(gap_cm=0.02, voltage_V=200.0)
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, 0.0, p)
    assert e.value.code == B.IT_ECUDA


def test_new_entry_points_reject_bad_arguments_without_a_gpu(L):
    import ctypes
    # a NULL context is refused before anything reaches the device
    xy = (ctypes.c_double * 2)(1e-3, 1e-3)
    one = (ctypes.c_double * 1)(1.0)
    assert L.it_deposit_tracks_angled(None, 1, xy, one, one, one) == B.IT_EINVAL
    n = ctypes.c_int64()
    assert L.it_dt_log(None, 0, None, None, None, ctypes.byref(n)) == B.IT_EINVAL
    # dt_ladder must be 0 or 1
    p = B.it_params_default(gap_cm=0.02, voltage_V=200.0, dt_ladder=2)
    with pytest.raises(B.ItError) as e:
        B.it_create(48, 48, 100, 2e-4, 0.0, p)
    assert e.value.code == B.IT_EINVAL


@pytest.mark.parametrize("space_charge", [0, 1])
def test_ladder_rule_matches_the_oracle(L, space_charge):
    # The library's rung (it_ladder_dt, the rule of it_run_to_completion) and
    # the oracle's ladder_dt are written independently.  Below the Eq.
    # (vNeum) cap a rung is dt times a power of two, so the two agree exactly;
    # at the cap they agree to the rounding of the two dt_vN evaluations.
    rng = np.random.default_rng(23)
    rungs = capped = 0
    for _ in range(4000):
        dx = 10.0 ** rng.uniform(-4.5, -3)
        nz = int(rng.integers(10, 400))
        V = float(rng.uniform(10, 500))
        scheme = int(rng.integers(0, 2))
        kappa = float(rng.choice([0.5, 0.25, 0.0625]))
        p = B.it_params_default(gap_cm=nz * dx, voltage_V=V, scheme=scheme, react_kappa=kappa,
                                space_charge=space_charge)
        cap = o.dt_von_neumann(dx, V, nz * dx, (1.73, 1.87), (0.037, 0.037), scheme)
        dt = cap * 10.0 ** rng.uniform(-4, 0)
        nmax = 10.0 ** rng.uniform(8, 15) if rng.random() < 0.95 else 0.0
        got = B.it_ladder_dt(p, dx, dt, nmax)
        want = o.ladder_dt(dt, nmax, 1.6e-6, cap, kappa, 1.87, bool(space_charge))
        if want < cap * (1 - 1e-12):
            assert got == want
            rungs += got > dt
        else:
            assert got == pytest.approx(want, rel=1e-14)
            capped += 1
    assert rungs > 500 and capped > 100
