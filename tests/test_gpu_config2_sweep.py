"""The pulsed workload's voltage sweep {50, 100, 200, 300, 400} V run to
completion on the GPU, each f held to the FP64 oracle's (Sec. Implementation:
a pulse run until the charge distributions are dragged apart; Sec. Results,
Fig. 4(a)).

The oracle values are stored in tests/golden/config2_sweep.json, written by
the script beside it from oracle/ only:

* full: the 256 x 256 x 400 grid itself (2000 tracks, LET log-uniform
  1-1000 keV/um), upwind drift, the doubling dt ladder at kappa = 1/16;
* section: a 64 x 64 x 400 section at the same track density with
  Lax-Wendroff drift and the ladder at kappa = 1/8 (the paper's scheme; at
  300 and 400 V it stops being finite in the oracle, and must on the GPU);
* section_fixed: the section with upwind drift and the fixed
  recombination-bound step (kappa = 0.5) at 200, 300 and 400 V.

Each GPU run takes the oracle's step count (the completion checks and the
ladder's rungs are decided independently on each side) and f within 1e-5.
"""
import json
import os

import pytest

from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "config2_sweep.json")


@pytest.fixture(scope="module")
def gold():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()
    with open(GOLD) as fh:
        return json.load(fh)


def section_tracks(V):
    return synth.uniform_tracks(1610067590 + int(V), 125, 64 * 5e-4, 64 * 5e-4, 1e-3, let="loguniform")


def run_gpu(nx, ny, nz, dx, V, tr, scheme, kappa, ladder):
    npk = B.it_peak_density(tr.let_keV_um, tr.b_cm)
    with B.Simulation(nx, ny, nz, dx, V, n_peak_cm3=npk, scheme=scheme, react_kappa=kappa,
                      dt_ladder=ladder) as g:
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        try:
            steps = g.run_to_completion(tol=1e-6, max_steps=10_000_000, check_every=64)
        except B.ItError as e:
            if e.code == B.IT_EUNSTABLE:
                return "unstable", None, None
            raise
        return "done", steps, g.tallies().f


def _check(ref, got):
    status, steps, f = got
    print(f"{ref['scheme']} {ref['voltage_V']:.0f} V kappa {ref['kappa']} ladder {ref['ladder']}: "
          f"GPU {status} {steps} {f} | oracle {ref['status']} {ref['steps']} {ref['f']}")
    assert status == ref["status"]
    if status == "done":
        assert steps == ref["steps"]
        assert abs(f - ref["f"]) <= 1e-5


@pytest.mark.parametrize("V", [50.0, 100.0, 200.0, 300.0, 400.0])
def test_full_grid_upwind_ladder_matches_oracle(gold, V):
    ref = next(r for r in gold["full"] if r["voltage_V"] == V)
    w = synth.pulsed_256x256x400(V)
    _check(ref, run_gpu(w.nx, w.ny, w.nz, w.dx_cm, V, synth.pulsed_tracks(w), B.IT_UPWIND, 0.0625, True))


@pytest.mark.parametrize("V", [50.0, 100.0, 200.0, 300.0, 400.0])
def test_section_lax_wendroff_ladder_matches_oracle(gold, V):
    ref = next(r for r in gold["section"] if r["voltage_V"] == V)
    _check(ref, run_gpu(64, 64, 400, 5e-4, V, section_tracks(V), B.IT_LAX_WENDROFF, 0.125, True))


@pytest.mark.parametrize("V", [200.0, 300.0, 400.0])
def test_section_upwind_fixed_step_matches_oracle(gold, V):
    ref = next(r for r in gold["section_fixed"] if r["voltage_V"] == V)
    _check(ref, run_gpu(64, 64, 400, 5e-4, V, section_tracks(V), B.IT_UPWIND, 0.5, False))
