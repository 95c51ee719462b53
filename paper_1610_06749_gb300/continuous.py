"""Continuous-beam workload run to steady state.

The 512 x 512 x 256 chamber section (dx = 8 um, gap 2.048 mm, 300 V, FP32,
periodic lateral faces) under Poisson arrivals of a 20 / 200 keV/um track
mixture (70 / 30 %, b = 10 um) at the given rates per cm^2 and second
(Sec. Implementation, "Distribution of ion tracks").  After a warm-up of two
ion transit times each run continues with it_run_to_steady_state: windows of
1000 steps until the departure efficiency of every ion that has left the
domain since the warm-up, Col / (Col + 2 Rec + Lost), moves by less than
1e-5 over a window that carried departures, or the step limit (a number of
transit times).  Reported: that efficiency with its batch-means standard
error, what stopped the run, the last window's own efficiency and the
cumulative f.  Upwind drift: at the recombination-bound time step
Lax-Wendroff's undershoots turn the recombination term into a source.
Every step runs in the CUDA solver; this module only generates the arrivals
(synth) and reports.

    python -m paper_1610_06749_gb300.continuous [rate ...]
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import binding as B
from . import synth


def run(rate_per_cm2_s: float, window: int = 1000, tol: float = 1e-5, transits: float = 100.0) -> dict:
    w = synth.continuous_512x512x256()
    npk = B.it_peak_density([200.0], [w.b_cm])
    with B.Simulation(w.nx, w.ny, w.nz, w.dx_cm, w.voltage_V, n_peak_cm3=npk, scheme=B.IT_UPWIND) as sim:
        dt = sim.tallies().dt_s
        E = w.voltage_V / w.gap_cm
        transit_steps = int(np.ceil(w.gap_cm / (min(synth.AIR["mu"]) * E * dt)))
        max_steps = int(transits * transit_steps) // window * window
        tr = synth.poisson_tracks(w.seed, rate_per_cm2_s, w.nx * w.dx_cm, w.ny * w.dx_cm, dt, max_steps, w.b_cm,
                                  synth.CONTINUOUS_LET)
        sim.autotune(trial_steps=8)
        if len(tr):
            sim.schedule(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm, tr.step)
        warm = (2 * transit_steps + window - 1) // window * window
        t0 = time.perf_counter()
        sim.step(warm)
        r = sim.run_to_steady_state(window_steps=window, tol=tol, max_steps=max_steps - warm)
        el = time.perf_counter() - t0
        t = sim.tallies()
        steps = warm + r["steps"]
        return {"workload": w.name, "rate_per_cm2_s": rate_per_cm2_s, "tracks_scheduled": len(tr),
                "tracks_arrived": int(np.sum(tr.step < steps)), "dt_s": dt, "transit_steps": transit_steps,
                "window_steps": window, "tol": tol, "f_ss": r["f_ss"], "f_ss_stderr": r["f_ss_stderr"],
                "f_last_window": r["f_window"], "windows": r["windows"],
                "stopped_by": "steady state" if r["stop"] == 0 else f"step limit ({transits:g} transits)",
                "steps": steps, "warmup_steps": warm, "seconds": el, "f_cumulative": t.f,
                "cell_updates_per_s": w.cells * steps / el, "launch": sim.launch()}


def main(argv=None):
    from . import build
    build.build()
    rates = [float(a) for a in (argv if argv is not None else sys.argv[1:])] or [1e5, 1e6, 1e7]
    out = []
    for r in rates:
        res = run(r)
        print(json.dumps(res), flush=True)
        out.append(res)
    return out


if __name__ == "__main__":
    main()
