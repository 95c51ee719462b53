"""Writes config2_sweep.json: FP64 oracle runs to completion of the pulsed
workload over the voltage sweep {50, 100, 200, 300, 400} V, the reference
that the GPU's runs of the same configurations are held to.

* full: the 256 x 256 x 400 grid itself (dx = 5 um, 2 mm gap, 2000 tracks,
  LET log-uniform 1-1000 keV/um, b = 10 um, periodic faces), upwind drift,
  the doubling dt ladder with kappa = 1/16, run until in-domain / released
  < 1e-6 (checked every 64 steps);
* section: a 64 x 64 x 400 section at the same track density (125 tracks,
  seed 1610067590 + V) run the same way with Lax-Wendroff drift and the
  ladder at kappa = 1/8 (a run whose state stops being finite is recorded
  with the step of the check that found it);
* section_fixed: the same section, upwind, the fixed recombination-bound
  step (kappa = 0.5), at 200, 300 and 400 V (the lower voltages take
  10^5 steps and more).

Calls only oracle/ and the seeded input generator.  Runs for about an hour
on eight cores.

    python tests/golden/make_config2_sweep.py [out.json]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.oracle as o  # noqa: E402
from paper_1610_06749_gb300 import synth  # noqa: E402

VOLTS = (50.0, 100.0, 200.0, 300.0, 400.0)


def section_tracks(V):
    return synth.uniform_tracks(1610067590 + int(V), 125, 64 * 5e-4, 64 * 5e-4, 1e-3, let="loguniform")


def one(nx, ny, nz, dx, V, tr, scheme, kappa, ladder):
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
    dt = o.dt_rule(dx, V, nz * dx, n_peak=npk, kappa=kappa, scheme=scheme)
    orc = o.Oracle(nx, ny, nz, dx, dt, voltage_V=V, scheme=scheme)
    t0 = time.time()
    try:
        orc.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        try:
            steps, done, log = orc.run_to_completion(tol=1e-6, check_every=64, ladder=ladder, kappa=kappa)
            t = orc.tallies()
            res = {"status": "done" if done else "step limit", "steps": int(steps), "f": t.f,
                   "rungs": len(log), "dt0_s": dt, "dt_end_s": t.dt_s}
        except FloatingPointError:
            res = {"status": "unstable", "steps": int(orc.tallies().steps), "f": None}
    finally:
        orc.close()
    res.update({"voltage_V": V, "kappa": kappa, "ladder": ladder,
                "scheme": "upwind" if scheme == o.SCHEME_UPWIND else "lax-wendroff",
                "oracle_seconds": round(time.time() - t0, 1)})
    print(json.dumps(res), flush=True)
    return res


def main():
    out_path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "config2_sweep.json")
    out = {"source": "FP64 oracle (oracle/iontracks_oracle.c), runs to completion (in-domain / released < 1e-6, "
                     "checked every 64 steps)", "full": [], "section": [], "section_fixed": []}
    for V in VOLTS:
        out["section"].append(one(64, 64, 400, 5e-4, V, section_tracks(V), o.SCHEME_LAX_WENDROFF, 0.125, True))
    for V in (400.0, 300.0, 200.0):
        out["section_fixed"].append(one(64, 64, 400, 5e-4, V, section_tracks(V), o.SCHEME_UPWIND, 0.5, False))
    for V in VOLTS:
        w = synth.pulsed_256x256x400(V)
        out["full"].append(one(w.nx, w.ny, w.nz, w.dx_cm, V, synth.pulsed_tracks(w), o.SCHEME_UPWIND, 0.0625, True))
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
