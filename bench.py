#!/usr/bin/env python
"""Throughput benchmark of the IonTracks transport step on GB300.

Workload: the pulsed-beam grid, 256 x 256 x 400 cells at dx = 5 um (2 mm
gap), FP32 densities with FP64 tallies, periodic lateral faces, 2000 tracks
per pulse at seeded uniform (x, y) with log-uniform LET 1-1000 keV/um and
b = 10 um, 200 V, single pulse.  One benchmark step is the first ``--seg``
explicit time steps (default 200) of a fresh single-pulse run: the state is
reset, the 2000-track pulse deposited, then the steps taken.
Metric: Gcell-updates/s (cells x time steps / s).

  value  -- device-timed (CUDA events on the library's stream), tracks resident in HBM
  e2e    -- through the public C API with host buffers: pinned track upload,
            deposit, steps, tally read-back, on the host clock
  roofline -- the step kernel: 16 algorithmic bytes per FP32 cell-update
            (read and write n+ and n-) / its average duration, against the
            measured HBM copy bandwidth
  cpu_baseline -- the FP64 CPU oracle on the host cores, bounded sample
  batched -- solves/s of a 256-simulation batch against one context per
            simulation, with the fixed step and with the doubling dt ladder
  time_to_solution -- the workload run to completion (upwind), fixed
            recombination-bound step against the dt ladder

``--impl reference`` times the oracle (the reference arm of this project) on
the same workload.  Under torchrun every rank runs an independent replica
(weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_CELL_UPDATE = 16          # FP32: read n+, n- once, write them once
FALLBACK_HBM_GBS = 6800.0
PROFILE = os.path.join(ROOT, "profiles", "step_zmarch_pulsed_256x256x400.json")


REPLICA_SEED_STRIDE = 7919


def replica_seed(seed, rank):
    """Seed of a rank's replica: every rank runs its own independent pulse
    (weak scaling, no data-path collective)."""
    return seed + REPLICA_SEED_STRIDE * rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device=None):
    """The largest x over the ranks: the job's time is its slowest rank's.
    device: where the reduction tensor lives (cuda for NCCL, cpu for gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Units all ranks processed, per second of the slowest rank."""
    return units_per_rank * ws / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in mp:
                v = mp[key]
                v = v.get("value", v) if isinstance(v, dict) else v
                return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_sha():
    """Hash of the sources of the step kernel's device code: it_zmarch.cu,
    it_tma.cuh, it_device.cuh and the device-side types of it_internal.cuh
    (the text before the host context struct, which the kernel never sees)."""
    h = hashlib.sha256()
    for name in ("it_zmarch.cu", "it_tma.cuh", "it_device.cuh", "it_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1610_06749_gb300", "csrc", name), "rb") as f:
            text = f.read()
        if name == "it_internal.cuh":
            text = text.split(b"\nstruct it_ctx {", 1)[0]
        h.update(text)
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel source has changed since it was captured."""
    try:
        with open(PROFILE) as f:
            prof = json.load(f)
        if prof.get("kernel_sha") == kernel_sha():
            return float(prof["dram_bytes_per_launch_full_size"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.tmp:
            return None
        try:
            rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.tmp.name)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(w, tracks, seconds):
    """Oracle Gcell-updates/s on the host cores, bounded sample of the workload."""
    import oracle.oracle as o
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    dt = o.dt_rule(w.dx_cm, w.voltage_V, w.gap_cm, n_peak=o.peak_track_density(tracks.let_keV_um, tracks.b_cm))
    O = o.Oracle(w.nx, w.ny, w.nz, w.dx_cm, dt, voltage_V=w.voltage_V)
    O.deposit(tracks.x_cm, tracks.y_cm, tracks.let_keV_um, tracks.b_cm)
    t0 = time.perf_counter()
    O.step(1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    O.step(n)
    el = time.perf_counter() - t0
    O.close()
    return w.cells * n / el / 1e9, int(os.environ.get("OMP_NUM_THREADS", cores)), n, el


def continuous_roofline(B, synth, dev, steps=500):
    """Step-kernel rate on the continuous-beam grid 512x512x256 (FP32, 1.07 GB
    of state with the ping-pong set): the Poisson arrivals of the first three
    steps at 3e9 tracks/(cm^2 s) deposited (a dense field), the launch shape
    autotuned, then `steps` graph-replayed steps timed with CUDA events on the
    library stream."""
    import torch
    w = synth.continuous_512x512x256()
    npk = B.it_peak_density([200.0], [w.b_cm])
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sim = B.Simulation(w.nx, w.ny, w.nz, w.dx_cm, w.voltage_V, n_peak_cm3=npk, torch_state=True)
    try:
        dt = sim.tallies().dt_s
        tr = synth.poisson_tracks(w.seed, 1e7 * 300, w.nx * w.dx_cm, w.ny * w.dx_cm, dt, 3, w.b_cm,
                                  synth.CONTINUOUS_LET)
        sim.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        sim.autotune(trial_steps=8)
        sim.step(64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        peak, kind = hbm_peak()
        ach = BYTES_PER_CELL_UPDATE * w.cells / t / 1e9
        return {"workload": w.name, "cells": w.cells, "kernel_us": t * 1e6,
                "gcell_updates_per_s": w.cells / t / 1e9, "achieved_GBs": ach, "peak_GBs": peak,
                "peak_kind": kind, "frac": ach / peak, "launch": sim.launch(), "tracks": len(tr)}
    finally:
        sim.close()


LADDER_KAPPA = 0.0625


def batched_vs_plain(B, synth, n_subset=16, tol=1e-6, check_every=64, scheme=None):
    """Solves/s of the 256-simulation batch (uneven grids 32^3 .. 128x128x200,
    one launch per step for all running simulations, CUDA-graph segments)
    against the plain one-context-per-simulation solver on the same GPU.
    The plain solver runs a subset (the first n_subset simulations); the batch
    is timed on that subset too, and on all 256.  Context creation is outside
    the timed regions; deposition, the batch autotuner (it_batch_autotune)
    and the run to completion are inside.
    Runs to completion use the upwind drift: at the recombination-bound time
    step the Courant number is small and Lax-Wendroff's undershoots make the
    explicit recombination term a source (it diverges, in the FP64 oracle
    too), while upwind stays positive."""
    import torch
    if scheme is None:
        scheme = B.IT_UPWIND
    descs = synth.batch_descriptors()
    tracks = [synth.batch_tracks(d) for d in descs]
    sims = []
    for d, tr in zip(descs, tracks):
        sims.append(dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], dx_cm=d["dx_cm"], voltage_V=d["voltage_V"],
                         n_peak_cm3=B.it_peak_density(tr.let_keV_um, tr.b_cm)))

    def run_batch(idx, ladder=False, kappa=0.5):
        bt = B.Batch([sims[q] for q in idx], scheme=scheme, dt_ladder=ladder, react_kappa=kappa)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, q in enumerate(idx):
            tr = tracks[q]
            bt.deposit(k, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.retime()                      # dt bound from each deposited peak (overlaps included)
        ta = time.perf_counter()
        tune_us = bt.autotune(trial_steps=8)
        ta = time.perf_counter() - ta
        launches = bt.run(tol=tol, check_every=check_every)
        el = time.perf_counter() - t0
        out = [bt.tallies(k) for k in range(len(idx))]
        bt.close()
        return el, out, launches, (ta, tune_us)

    t_all, tal_all, launches, tune = run_batch(list(range(len(sims))))
    # the same 256 simulations with the doubling dt ladder of the runs to completion at
    # kappa = 1/16, judged against the fixed step at the same kappa (every step of both keeps
    # alpha dt n_max <= kappa).  The fixed step at kappa = 0.5 is itself off by up to 1.5e-2 on
    # the simulations that finish in a few dozen steps, so it is no reference for 1e-3.
    t_lad, tal_lad, launches_lad, tune_lad = run_batch(list(range(len(sims))), ladder=True, kappa=LADDER_KAPPA)
    t_fk, tal_fk, launches_fk, _ = run_batch(list(range(len(sims))), ladder=False, kappa=LADDER_KAPPA)
    df_lad = max(abs(a.f - b.f) for a, b in zip(tal_lad, tal_fk))
    df_k05 = max(abs(a.f - b.f) for a, b in zip(tal_all, tal_fk))
    sub = list(range(n_subset))
    t_bsub, tal_bsub, _, _ = run_batch(sub)
    ctxs = [B.Simulation(sims[q]["nx"], sims[q]["ny"], sims[q]["nz"], sims[q]["dx_cm"], sims[q]["voltage_V"],
                         n_peak_cm3=sims[q]["n_peak_cm3"], scheme=scheme) for q in sub]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f_plain = []
    for q, g in zip(sub, ctxs):
        tr = tracks[q]
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.retime()
        g.run_to_completion(tol=tol, check_every=check_every)
        f_plain.append(g.tallies().f)
    t_plain = time.perf_counter() - t0
    for g in ctxs:
        g.close()
    df = max(abs(a.f - b) for a, b in zip(tal_bsub, f_plain))
    cell_updates = sum(sims[q]["nx"] * sims[q]["ny"] * sims[q]["nz"] * tal_all[q].steps for q in range(len(sims)))
    cell_updates_lad = sum(sims[q]["nx"] * sims[q]["ny"] * sims[q]["nz"] * tal_lad[q].steps for q in range(len(sims)))
    return {"sims": len(sims), "solves_per_s": len(sims) / t_all, "seconds": t_all, "step_launches": launches,
            "autotune_s": tune[0], "autotuned_us_per_step": tune[1],
            # one batched step with every simulation active (the autotuner's best time): the
            # per-step rate before simulations finish and the tail leaves SMs idle
            "full_occupancy_Gcell_updates_per_s": sum(q["nx"] * q["ny"] * q["nz"] for q in sims) / tune[1] / 1e3,
            "full_occupancy_hbm_frac": BYTES_PER_CELL_UPDATE * sum(q["nx"] * q["ny"] * q["nz"] for q in sims)
                                       / tune[1] / 1e3 / hbm_peak()[0],
            "Gcell_updates_per_s": cell_updates / t_all / 1e9,
            "Gcell_updates_per_s_after_autotune": cell_updates / (t_all - tune[0]) / 1e9,
            "subset": n_subset, "subset_batched_solves_per_s": n_subset / t_bsub,
            "subset_plain_solves_per_s": n_subset / t_plain,
            "speedup_vs_plain": (n_subset / t_bsub) / (n_subset / t_plain),
            "max_abs_df_vs_plain": df, "df_bound": 1e-3, "scheme": "upwind" if scheme == B.IT_UPWIND else "lax-wendroff",
            # the ladder's speedup is reported only when its answers stay within df_bound of the
            # fixed-step batch; otherwise the line says so instead of giving a rate
            "ladder": {"kappa": LADDER_KAPPA, "step_launches": launches_lad,
                       "fixed_dt_same_kappa": {"seconds": t_fk, "step_launches": launches_fk,
                                               "solves_per_s": len(sims) / t_fk},
                       "max_abs_df_vs_fixed_dt_same_kappa": df_lad, "within_df_bound": df_lad <= 1e-3,
                       "fixed_kappa_0.5_max_abs_df_vs_kappa_1/16": df_k05,
                       "solves_per_s": len(sims) / t_lad if df_lad <= 1e-3 else None,
                       "seconds": t_lad, "autotune_s": tune_lad[0],
                       # cell-updates over the run after the autotuner, against the
                       # full-occupancy step: how much of the run the tail leaves idle
                       "Gcell_updates_per_s_after_autotune": cell_updates_lad / (t_lad - tune_lad[0]) / 1e9,
                       "speedup_vs_fixed_dt_same_kappa": t_fk / t_lad if df_lad <= 1e-3 else None,
                       "speedup_vs_fixed_dt_kappa_0.5": t_all / t_lad if df_lad <= 1e-3 else None}}


def time_to_solution(V):
    """The benchmark's pulsed workload run to completion (upwind), with the
    fixed recombination-bound step and with the doubling dt ladder."""
    from paper_1610_06749_gb300 import time_to_solution as T
    from paper_1610_06749_gb300 import binding as B
    fixed = T.run(V, B.IT_UPWIND, 0.5, False)
    lad = T.run(V, B.IT_UPWIND, 0.0625, True)
    keep = ("kappa", "status", "steps", "seconds", "f", "rungs")
    return {"workload": fixed["workload"], "scheme": "upwind", "fixed_dt": {k: fixed[k] for k in keep},
            "ladder": {k: lad[k] for k in keep}, "speedup": fixed["seconds"] / lad["seconds"],
            "abs_df": abs(fixed["f"] - lad["f"]) if fixed["f"] is not None and lad["f"] is not None else None}


def surrogate_vs_plain(n_train=48000, n_test=2000, epochs=2000, plain_sample=40):
    """The surrogate ensemble (trained on batched-solver runs of the
    surrogate workload) answering held-out configurations, falling back to the
    solver where its members disagree beyond the calibrated gate, against the
    batched and the plain solver alone.  The single-pulse half of the draws
    (about 24000 training and 1000 held-out configurations; trains of pulses
    carry ~25x the solver work); the full 20k/2k study,
    trains included, is `python -m paper_1610_06749_gb300.surrogate`.  The
    gains are reported only while the accepted answers meet the 99 %
    coverage within 1e-3."""
    from paper_1610_06749_gb300 import surrogate as S
    out = S.main(["--train", str(n_train), "--test", str(n_test), "--epochs", str(epochs),
                  "--plain-sample", str(plain_sample), "--single-pulse", "--val-frac", "0.15"], quiet=True)
    return out


def run_reference(args, ws, rank):
    from paper_1610_06749_gb300 import synth
    import oracle.oracle as o
    if rank != 0:
        return
    w = synth.pulsed_256x256x400(args.voltage)
    tracks = synth.pulsed_tracks(w)
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    dt = o.dt_rule(w.dx_cm, w.voltage_V, w.gap_cm, n_peak=o.peak_track_density(tracks.let_keV_um, tracks.b_cm))
    O = o.Oracle(w.nx, w.ny, w.nz, w.dx_cm, dt, voltage_V=w.voltage_V)
    O.deposit(tracks.x_cm, tracks.y_cm, tracks.let_keV_um, tracks.b_cm)
    for _ in range(args.warmup):
        O.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(1)
    el = time.perf_counter() - t0
    val = w.cells * args.steps / el / 1e9
    sample = (f"FP64 oracle, {args.steps} explicit steps of the {w.nx}x{w.ny}x{w.nz} pulsed grid after one "
              f"2000-track pulse (one oracle step per benchmark step)")
    line = {"impl": "reference", "metric": "Gcell-updates/s", "value": val, "unit": "Gcell-updates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "cells": w.cells, "tracks_per_pulse": 2000},
            "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1610_06749_gb300 import build as libbuild
    libbuild.build()
    from paper_1610_06749_gb300 import binding as B
    from paper_1610_06749_gb300 import synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = synth.pulsed_256x256x400(args.voltage)
    w.seed = replica_seed(w.seed, rank)            # independent replica per rank
    tracks = synth.pulsed_tracks(w)
    ntr = len(tracks)
    npk = B.it_peak_density(tracks.let_keV_um, tracks.b_cm)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sim = B.Simulation(w.nx, w.ny, w.nz, w.dx_cm, w.voltage_V, n_peak_cm3=npk, torch_state=True)
    # native autotuner (below): fastest launch shape of the step kernel on
    # this grid, timed on the deposited pulse (the state is restored)
    packed = np.stack([tracks.x_cm, tracks.y_cm, tracks.let_keV_um, tracks.b_cm], axis=1)
    d_tracks = torch.from_numpy(np.ascontiguousarray(packed)).to(dev)
    xy_host = np.ascontiguousarray(np.stack([tracks.x_cm, tracks.y_cm], axis=1))
    torch.cuda.synchronize()          # d_tracks was written on torch's default stream
    B.it_deposit_tracks_device(sim.h, ntr, d_tracks.data_ptr())
    if args.launch:
        ty, cps, st, grid = (int(v) for v in args.launch.split(","))
        sim.set_launch(B.IT_KERNEL_ZMARCH, ty, cps, st, grid)
        tune_us = None
    else:
        tune_us = sim.autotune(trial_steps=8)
    sim.reset()
    launch = sim.launch()
    cells, seg = w.cells, args.seg

    def maxover(x):
        return max_over_ranks(x, ws, dev)

    def dev_step():
        sim.reset()
        B.it_deposit_tracks_device(sim.h, ntr, d_tracks.data_ptr())
        sim.step(seg)

    # ---- device-timed throughput (inputs resident in HBM) ----
    for _ in range(args.warmup):
        dev_step()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            dev_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    t_dev = maxover(ev0.elapsed_time(ev1) / 1e3)
    clocks = clk.summary()

    # ---- step-kernel duration (graph replays, no deposits), same stream ----
    nk = max(2 * seg, 1000)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.step(64)
    torch.cuda.synchronize()
    k0.record(stream)
    sim.step(nk)
    k1.record(stream)
    torch.cuda.synchronize()
    t_kernel = k0.elapsed_time(k1) / 1e3 / nk

    # the temporal-blocking variant (two steps per launch) on the same state,
    # for the record of what the autotuner weighed
    tb2 = None
    try:
        with torch.cuda.stream(stream):
            sim2 = B.Simulation(w.nx, w.ny, w.nz, w.dx_cm, w.voltage_V, n_peak_cm3=npk, torch_state=True,
                                kernel=B.IT_KERNEL_ZMARCH2)
        B.it_deposit_tracks_device(sim2.h, ntr, d_tracks.data_ptr())
        sim2.step(64)
        torch.cuda.synchronize()
        k0.record(stream)
        sim2.step(nk)
        k1.record(stream)
        torch.cuda.synchronize()
        tb2 = {"kernel": "step_zmarch2_kernel (two steps per launch)", "launch": sim2.launch(),
               "us_per_step": k0.elapsed_time(k1) * 1e3 / nk}
        sim2.close()
    except Exception as e:   # a grid the two-step kernel cannot tile
        tb2 = {"unavailable": str(e)}

    # ---- end to end through the public API with host buffers ----
    def e2e_step():
        sim.reset()
        B.it_deposit_tracks(sim.h, xy_host, tracks.let_keV_um, tracks.b_cm)   # pinned staging H2D
        sim.step(seg)
        return sim.tallies()                                                    # D2H of the tallies
    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = e2e_step()
    t_e2e = maxover(time.perf_counter() - t0)
    barrier(ws)

    total_updates = cells * seg * args.steps * ws
    value = whole_job_rate(cells * seg * args.steps, ws, t_dev) / 1e9
    e2e_value = whole_job_rate(cells * seg * args.steps, ws, t_e2e) / 1e9
    peak, peak_kind = hbm_peak()
    achieved = BYTES_PER_CELL_UPDATE * cells / t_kernel / 1e9
    traffic = ncu_traffic()

    cont = None
    if rank == 0 and not args.no_continuous:
        cont = continuous_roofline(B, synth, dev)
    batched = None
    if not args.no_batched:
        batched = batched_vs_plain(B, synth)
    sur = None
    if not args.no_surrogate and rank == 0:
        sur = surrogate_vs_plain()
    tts = None
    if not args.no_time_to_solution and rank == 0:
        tts = time_to_solution(args.voltage)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            rate, cores, n, el = cpu_oracle_rate(w, tracks, args.cpu_seconds)
            cpu = {"value": rate, "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
                   "sample": f"FP64 oracle, {n} explicit steps of the {w.nx}x{w.ny}x{w.nz} pulsed grid after "
                             f"one 2000-track pulse ({el:.1f} s)"}
        line = {
            "metric": "Gcell-updates/s", "value": value, "unit": "Gcell-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "dx_um": w.dx_cm * 1e4,
                       "tracks_per_pulse": ntr, "time_steps_per_step": seg, "voltage_V": w.voltage_V,
                       "tallies": "f64", "kernel": {B.IT_KERNEL_ZMARCH: "zmarch", B.IT_KERNEL_ZMARCH2: "zmarch2"}.get(
                           launch["kernel"], "simple"),
                       "launch": launch, "autotune_us_per_step": tune_us, "l2": "inputs larger than L2 (210 MB state read per time step)",
                       "parallelism": f"replicas{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         # two steps per launch read and write the state once per two steps:
                         # 16 B per cell-update is then an effective figure
                         "effective": launch["kernel"] == B.IT_KERNEL_ZMARCH2,
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "step_zmarch2_kernel" if launch["kernel"] == B.IT_KERNEL_ZMARCH2 else "step_zmarch_kernel",
                         "kernel_us": t_kernel * 1e6,
                         "bytes_per_launch": BYTES_PER_CELL_UPDATE * cells},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": ntr * 4 * 8,
                    "d2h_bytes_per_step": 17 * 8},
            # per benchmark step: 4 deposit kernels + the step launches (two steps
            # per launch with the two-step kernel, the odd one on the simple kernel)
            "gpu_launches": args.steps * (4 + (seg // 2 + seg % 2 if launch["kernel"] == B.IT_KERNEL_ZMARCH2 else seg)),
            "temporal_blocking_2": tb2,
            "clocks": clocks,
            "f_last": t.f,
            "roofline_continuous_512x512x256": cont,
            "batched": batched,
            "surrogate": sur,
            "time_to_solution": tts,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30, help="benchmark steps (pulse periods) timed")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seg", type=int, default=200, help="explicit time steps per benchmark step")
    ap.add_argument("--voltage", type=float, default=200.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain solves/s measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate-vs-plain solves/s measurement")
    ap.add_argument("--no-continuous", action="store_true", help="skip the 512x512x256 step-kernel roofline line")
    ap.add_argument("--no-time-to-solution", action="store_true",
                    help="skip the run to completion with a fixed step and with the dt ladder")
    ap.add_argument("--launch", default="", help="fixed z-march shape TY,ctas_per_sm,stages,grid (skips the autotuner)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
