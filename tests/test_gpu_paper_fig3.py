"""The paper's Fig. 3 comparison on its own parameters, with the CUDA solver.

Single tracks of Table 1 (iron, neon, carbon) with the Table 2 ion constants,
electrode spacing 2 mm, dx = b/20 and Lx = Ly = 10 b (the grid rule of
Sec. Stability and accuracy), absorbing lateral faces, Lax-Wendroff drift,
run to completion at three field strengths:

* Fig. 3(a): tracks parallel to the field against Eq. (Jaffe_noangle);
* Fig. 3(b): the neon track parallel to the electrodes (theta = pi/2, a
  track along x at mid-gap, periodic in x) against Eq. (angle).

The figures print no values, so the table is the reproduction; run with
``-s`` to print it.  D and mu in the closed forms are the means of the two
species (Sec. "The Jaffe theory", the text under Eq. Jaffe_noangle).

Jaffe's closed forms describe initial recombination, so each run is
compared through f_rec = 1 - recombined/released (per species), the
efficiency without the ions lost through the lateral faces; f itself
(collected/released) is compared too wherever those losses stay below a
tenth of the recombined fraction.  At 300 V/cm the ions diffuse about 65 um sideways
during the 0.5 ms transit, more than the 5 b half-width of the carbon box
(52 um), so there the 10 b box of the grid rule loses ions at its faces
(the paper asks for boxes large enough that this does not happen).
"""
import json
import math
import os

import pytest

import oracle.oracle as o
from paper_1610_06749_gb300 import binding as B

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")
FIELDS = (300.0, 1000.0, 3000.0)


@pytest.fixture(scope="module")
def paper():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()
    g = json.load(open(GOLDEN))
    t2 = g["table2_ion_constants"]
    mu = (t2["mu_plus_cm2_Vs"], t2["mu_minus_cm2_Vs"])
    D = (t2["D_plus_cm2_s"], t2["D_minus_cm2_s"])
    return g["table1_track_parameters"], mu, D, t2["alpha_cm3_s"], g["fig2_grid_rule"]


def _run(nx, ny, nz, dx, E, mu, D, alpha, let, b, theta, lateral):
    V = E * nz * dx
    npk = B.it_peak_density([let], [b])
    with B.Simulation(nx, ny, nz, dx, V, mu=mu, D=D, alpha=alpha, lateral_bc=lateral, n_peak_cm3=npk) as g:
        x, y = 0.5 * nx * dx, 0.5 * ny * dx
        if theta == 0.0:
            g.deposit([x], [y], [let], [b])
        else:
            g.deposit_angled([x], [y], [let], [b], [theta])
        g.run_to_completion(tol=1e-6, max_steps=2_000_000, check_every=256)
        t = g.tallies()
        rel = t.released[0]
        return t.f, 1.0 - t.recombined / rel, t.lost_lateral.sum() / t.released.sum()


@pytest.mark.parametrize("ion", ["iron", "neon", "carbon"])
def test_fig3a_parallel_tracks_against_jaffe(paper, ion):
    tracks, mu, D, alpha, rule = paper
    p = tracks[ion]
    b = p["b_um"] * 1e-4
    dx = b * rule["dx_over_b"]
    n_lat = int(round(rule["Lx_over_b"] / rule["dx_over_b"]))
    nz = int(round(0.2 / dx))
    gap = nz * dx
    rows = []
    for E in FIELDS:
        f, frec, lost = _run(n_lat, n_lat, nz, dx, E, mu, D, alpha, p["LET_keV_um"], b, 0.0, B.IT_ABSORBING)
        fj = o.jaffe_parallel(p["LET_keV_um"], b, gap, E, 0.5 * (mu[0] + mu[1]), 0.5 * (D[0] + D[1]), alpha)
        rows.append((E, f, frec, lost, fj))
        print(f"\nFig3a {ion:6s} E {E:6.0f} V/cm  f {f:.5f}  f_rec {frec:.5f}  lost {lost:.2e}  Jaffe {fj:.5f}  "
              f"f_rec - f_J {frec - fj:+.2e}  (1 - f_J {1 - fj:.4f})")
    # measured: |f_rec - f_J| / (1 - f_J) = 4.5 % (iron, 300 V/cm) and 0.3-2.6 %
    # elsewhere; the bound is 10 % of the recombined fraction
    for E, f, frec, lost, fj in rows:
        assert abs(frec - fj) <= 0.1 * (1.0 - fj) + 5e-4
        if lost < 0.1 * (1.0 - fj):
            assert abs(f - fj) <= 0.1 * (1.0 - fj) + 5e-4


def test_fig3b_neon_parallel_to_the_electrodes_against_jaffe_angle(paper):
    tracks, mu, D, alpha, rule = paper
    p = tracks["neon"]
    b = p["b_um"] * 1e-4
    dx = b * rule["dx_over_b"]
    ny = int(round(rule["Lx_over_b"] / rule["dx_over_b"]))
    nz = int(round(0.2 / dx))
    for E in FIELDS:
        f, frec, _ = _run(4, ny, nz, dx, E, mu, D, alpha, p["LET_keV_um"], b, math.pi / 2, B.IT_PERIODIC)
        fj = o.jaffe_angle(p["LET_keV_um"], b, E, math.pi / 2, 0.5 * (mu[0] + mu[1]), 0.5 * (D[0] + D[1]), alpha)
        print(f"\nFig3b neon pi/2 E {E:6.0f} V/cm  f {f:.6f}  f_rec {frec:.6f}  Jaffe {fj:.6f}  f - f_J {f - fj:+.2e}  "
              f"(1 - f_J {1 - fj:.5f})")
        # measured 1.4-2.8 % of the recombined fraction
        assert abs(f - fj) <= 0.1 * (1.0 - fj) + 5e-6
