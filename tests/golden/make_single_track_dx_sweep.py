"""Writes single_track_dx_sweep.json: the FP64 oracle's collection efficiency
of the single-track workload (LET 100 keV/um, b = 10 um, 200 V over a 200 um
gap, a 96 um square section with absorbing faces, the track along z at the
centre) at dx = b/5, b/10 and b/20, each run to completion (in-domain /
released < 1e-9, checked every 32 steps), beside Jaffe's Eq. (Jaffe_noangle)
for the same track.  Calls only oracle/.  The b/20 run takes about two
minutes on eight cores.

    python tests/golden/make_single_track_dx_sweep.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.oracle as o  # noqa: E402

LET, B_CM, V, GAP, SIDE = 100.0, 1e-3, 200.0, 0.02, 96e-4
MU, D, ALPHA = (1.73, 1.87), 0.037, 1.6e-6


def case(k):
    dx = B_CM / k
    nx, nz = int(round(SIDE / dx)), int(round(GAP / dx))
    dt = o.dt_rule(dx, V, GAP, n_peak=o.peak_track_density([LET], [B_CM]))
    orc = o.Oracle(nx, nx, nz, dx, dt, voltage_V=V, lateral_bc=o.LATERAL_ABSORBING)
    try:
        orc.deposit([0.5 * nx * dx], [0.5 * nx * dx], [LET], [B_CM])
        steps, done, _ = orc.run_to_completion(tol=1e-9, check_every=32)
        assert done
        t = orc.tallies()
        return {"b_over_dx": k, "dx_cm": dx, "nx": nx, "ny": nx, "nz": nz, "dt_s": dt, "steps": int(steps),
                "f": t.f, "recombined_fraction": t.recombined / t.released[0],
                "lost_lateral_fraction": float(t.lost_lateral.sum() / t.released.sum())}
    finally:
        orc.close()


def main():
    fj = o.jaffe_parallel(LET, B_CM, GAP, V / GAP, 0.5 * (MU[0] + MU[1]), D, ALPHA)
    out = {"source": "FP64 oracle (oracle/iontracks_oracle.c) run to completion; Jaffe: Eq. (Jaffe_noangle) "
                     "with the species means of mu and D",
           "LET_keV_um": LET, "b_cm": B_CM, "voltage_V": V, "gap_cm": GAP, "side_cm": SIDE,
           "f_jaffe": fj, "runs": [case(k) for k in (5, 10, 20)]}
    with open(os.path.join(HERE, "single_track_dx_sweep.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
