"""Pulsed runs to completion with a fixed time step and with the dt ladder.

The 256 x 256 x 400 pulsed workload (2000 tracks, LET log-uniform 1-1000
keV/um, b = 10 um, dx = 5 um, FP32, periodic lateral faces) is run until
the ions left in the domain are below 1e-6 of the released ones (Sec.
Implementation: the tracks are dragged apart), checked every 64 steps, for
each voltage, drift scheme and reaction bound kappa:

* fixed: dt = min(dt_vN, kappa / (alpha n_peak)) for the whole run;
* ladder: the same start, then at every check dt rises to the largest
  power-of-two multiple still within kappa / (alpha n_max) of the current
  state, capped at the Eq. (vNeum) step (it_run_to_completion with
  dt_ladder = 1).

Reported per run: steps, wall seconds (the solver on the GPU, checks
included), f, the simulated time and the number of rungs; a run whose state
stopped being finite is reported as unstable.  Every step runs in the CUDA
solver; this module only sets the runs up and reports.

    python -m paper_1610_06749_gb300.time_to_solution [V ...]
    python -m paper_1610_06749_gb300.time_to_solution sweep
"""
from __future__ import annotations

import json
import sys
import time

from . import binding as B
from . import synth


def run(V: float, scheme: int, kappa: float, ladder: bool, max_steps: int = 2_000_000) -> dict:
    w = synth.pulsed_256x256x400(V)
    tr = synth.pulsed_tracks(w)
    npk = B.it_peak_density(tr.let_keV_um, tr.b_cm)
    out = {"workload": w.name, "voltage_V": V, "scheme": "upwind" if scheme == B.IT_UPWIND else "lax-wendroff",
           "kappa": kappa, "mode": "ladder" if ladder else "fixed"}
    with B.Simulation(w.nx, w.ny, w.nz, w.dx_cm, V, n_peak_cm3=npk, scheme=scheme, react_kappa=kappa,
                      dt_ladder=ladder) as sim:
        sim.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        dt0 = sim.tallies().dt_s
        t0 = time.perf_counter()
        status = "done"
        try:
            steps = sim.run_to_completion(tol=1e-6, max_steps=max_steps, check_every=64)
        except B.ItError as e:
            status = {B.IT_EUNSTABLE: "unstable", B.IT_ETIMEOUT: "step limit"}.get(e.code, str(e))
            steps = None
        el = time.perf_counter() - t0
        t = sim.tallies()
        out.update({"status": status, "steps": t.steps if steps is None else steps, "seconds": el,
                    "f": t.f if status == "done" else None, "t_s": t.t_s, "dt0_s": dt0, "dt_end_s": t.dt_s,
                    "rungs": len(sim.dt_log())})
    return out


def sweep(volts=(50.0, 100.0, 200.0, 300.0, 400.0)):
    """The pulsed workload's voltage sweep run to completion: upwind with the
    fixed recombination-bound step (kappa = 0.5), upwind with the ladder at
    kappa = 1/16, and the paper's Lax-Wendroff drift with the ladder at
    kappa = 1/8."""
    out = []
    for V in volts:
        for scheme, kappa, ladder in ((B.IT_UPWIND, 0.5, False), (B.IT_UPWIND, 0.0625, True),
                                      (B.IT_LAX_WENDROFF, 0.125, True)):
            r = run(V, scheme, kappa, ladder, max_steps=400_000)
            print(json.dumps(r), flush=True)
            out.append(r)
    return out


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if argv and argv[0] == "sweep":
        return sweep()
    volts = [float(a) for a in argv] or [50.0, 200.0]
    for V in volts:
        # upwind: fixed steps down to kappa = 0.125 give the convergence in dt
        for kappa in (0.5, 0.25, 0.125):
            print(json.dumps(run(V, B.IT_UPWIND, kappa, False)), flush=True)
        for kappa in (0.5, 0.25, 0.125, 0.0625):
            print(json.dumps(run(V, B.IT_UPWIND, kappa, True)), flush=True)
        # Lax-Wendroff: one fixed run, bounded (at the recombination-bound
        # step its undershoots can make the reaction term a source)
        print(json.dumps(run(V, B.IT_LAX_WENDROFF, 0.5, False, max_steps=300_000)), flush=True)
        for kappa in (0.5, 0.25, 0.125, 0.0625):
            print(json.dumps(run(V, B.IT_LAX_WENDROFF, kappa, True)), flush=True)


if __name__ == "__main__":
    main()
