"""The batched workload at full occupancy: many uneven simulations advanced by
one launch per step.

The first --sims simulations of synth.batch_descriptors() (nx, ny 32-128,
nz 32-200, dx 2-8 um, 50-400 V, 1-500 tracks of one LET and b each) are
created as one batch, their tracks deposited, every dt retimed from the
deposited peak, the launch shape chosen by the native autotuner
(it_batch_autotune), and then --steps steps run with every simulation still
active: at the fixed recombination-bound step the shortest simulation of
the set needs 128 steps.

Reported: the autotuner's best time per step, the host-timed run of the
steps (CUDA-graph segments of 64 steps, completion checks included), the
cell-updates per second of each, and the algorithmic bandwidth at 16 bytes
per FP32 cell update (read and write n+ and n-).  Every step runs in the
CUDA solver; this module only sets the batch up and reports.

    python -m paper_1610_06749_gb300.batched [--sims N] [--steps M]
"""
from __future__ import annotations

import argparse
import json
import time

from . import binding as B
from . import synth

BYTES_PER_CELL_UPDATE = 16


def full_occupancy(n_sims: int = 256, steps: int = 64, scheme: int = B.IT_UPWIND) -> dict:
    descs = synth.batch_descriptors()[:n_sims]
    tracks = [synth.batch_tracks(d) for d in descs]
    sims = [dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], dx_cm=d["dx_cm"], voltage_V=d["voltage_V"],
                 n_peak_cm3=B.it_peak_density(tr.let_keV_um, tr.b_cm)) for d, tr in zip(descs, tracks)]
    cells = sum(s["nx"] * s["ny"] * s["nz"] for s in sims)
    with B.Batch(sims, scheme=scheme) as bt:
        for k, tr in enumerate(tracks):
            bt.deposit(k, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.retime()
        tune_us = bt.autotune(trial_steps=8)
        t0 = time.perf_counter()
        launches = bt.run(tol=0.0, max_steps=steps, check_every=64)
        el = time.perf_counter() - t0
        still = sum(1 for k in range(len(sims)) if bt.tallies(k).steps >= steps)
    run_us = el / max(launches, 1) * 1e6
    return {"sims": len(sims), "cells": cells, "steps": launches, "sims_active_throughout": still,
            "autotuned_us_per_step": tune_us,
            "autotuned_Gcell_updates_per_s": cells / tune_us / 1e3,
            "autotuned_GBs": BYTES_PER_CELL_UPDATE * cells / tune_us / 1e3,
            "run_us_per_step": run_us,
            "run_Gcell_updates_per_s": cells / run_us / 1e3,
            "run_GBs": BYTES_PER_CELL_UPDATE * cells / run_us / 1e3}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sims", type=int, default=256, help="the first N simulations of the batched workload")
    ap.add_argument("--steps", type=int, default=64, help="steps run after the autotuner (a multiple of 64)")
    a = ap.parse_args(argv)
    print(json.dumps(full_occupancy(a.sims, a.steps)))


if __name__ == "__main__":
    main()
