"""Surrogate workflow: solver-generated data, ensemble training, prediction
with a fall-back to the solver.

Orchestration only -- every solve runs in the CUDA solver (batched or one
context per configuration), every training and inference step in the CUDA
network kernels; this module moves arrays between them.

A configuration (synth.surrogate_configs) is released as one pulse, or a
train of 4 identical pulses; its first time step is the automatic rule with
the recombination bound of peak_bound (a smooth function of the inputs),
after the last pulse the doubling dt ladder at kappa = 1/16 raises it, and a
train's period is rounded to a whole number of 64-step check intervals (the
period actually simulated is the sixth network input).  Runs to completion
use the upwind drift (stable at the recombination-bound time step, where
Lax-Wendroff diverges).
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B
from . import synth

CHECK = synth.SURROGATE_CHECK
TOL = 1e-6
# runs to completion: the doubling dt ladder from the recombination bound at
# kappa = 1/16 (time-discretization error ~1e-5 in f on the pulsed workload,
# against ~4e-3 for a fixed step at kappa = 0.5, and 10x fewer steps)
LADDER = True
KAPPA = 0.0625


def peak_bound(c) -> float:
    """Density bound of a configuration for its recombination time step: the
    single-track centre density N0 / (pi b^2) (Eqs. linear_density, Gaussian)
    plus the uniform density of its tracks spread over the section, times the
    pulse count.  A smooth function of the inputs (the largest density of the
    deposited state is not: it jumps as tracks overlap on the grid), so the
    time-discretization error of f varies smoothly with the inputs too."""
    single = B.it_peak_density([c["let"]], [c["b_cm"]])
    area = (c["nx"] * c["dx_cm"]) * (c["ny"] * c["dx_cm"])
    return c["pulses"] * single * (1.0 + c["n_tracks"] * np.pi * c["b_cm"] ** 2 / area)


def _desc(c):
    return dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], dx_cm=c["dx_cm"], voltage_V=c["voltage_V"],
                n_peak_cm3=peak_bound(c))


def est_steps(c, kappa=KAPPA) -> float:
    """Rough step count of a configuration's run: the pulses of a train at
    the first time step, then one ion transit at it (the ladder shortens the
    rest).  Only orders the configurations into batches."""
    p = B.it_params_default(gap_cm=c["gap_cm"], voltage_V=c["voltage_V"], scheme=B.IT_UPWIND, react_kappa=kappa,
                            n_peak_cm3=peak_bound(c))
    dt = B.it_auto_dt(p, c["dx_cm"])
    transit = c["gap_cm"] ** 2 / (min(synth.AIR["mu"]) * c["voltage_V"])
    return ((c["pulses"] - 1) * c["period_s"] + transit) / dt


def solve_batch(cfgs, chunk=2048, ladder=LADDER, kappa=KAPPA):
    """f of every configuration with the batched solver.  Returns (f, dt,
    period_steps) arrays (dt: the initial time step).  A batch runs until its
    slowest simulation completes, so the configurations are batched in the
    order of their estimated step counts: the long trains share batches
    instead of holding up every batch."""
    n = len(cfgs)
    f = np.full(n, np.nan)
    dt = np.zeros(n)
    per = np.zeros(n, dtype=np.int64)
    order = np.argsort([est_steps(c, kappa) for c in cfgs], kind="stable") if n > chunk else np.arange(n)
    for a in range(0, n, chunk):
        idx = order[a:a + chunk]
        part = [cfgs[i] for i in idx]
        with B.Batch([_desc(c) for c in part], scheme=B.IT_UPWIND, dt_ladder=ladder, react_kappa=kappa) as bt:
            for k, c in enumerate(part):
                tr = synth.surrogate_tracks(c)
                bt.deposit(k, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
            for k, c in enumerate(part):
                dt[idx[k]] = bt.tallies(k).dt_s
                if c["pulses"] > 1:
                    p = max(1, int(round(c["period_s"] / dt[idx[k]] / CHECK))) * CHECK
                    per[idx[k]] = p
                    bt.set_pulses(k, c["pulses"], p)
            bt.run(tol=TOL, check_every=CHECK)
            for k in range(len(part)):
                f[idx[k]] = bt.tallies(k).f
    return f, dt, per


def solve_plain(c, dt, period_steps, ladder=LADDER, kappa=KAPPA):
    """f of one configuration with one solver context (the method without the
    surrogate), from the given initial time step and pulse period."""
    with B.Simulation(c["nx"], c["ny"], c["nz"], c["dx_cm"], c["voltage_V"], dt_s=dt,
                      scheme=B.IT_UPWIND, dt_ladder=ladder, react_kappa=kappa) as g:
        tr = synth.surrogate_tracks(c)
        if c["pulses"] > 1:
            n = len(tr)
            steps = np.repeat(np.arange(c["pulses"], dtype=np.int64) * period_steps, n)
            rep = lambda a: np.tile(a, c["pulses"])
            g.schedule(rep(tr.x_cm), rep(tr.y_cm), rep(tr.let_keV_um), rep(tr.b_cm), steps)
        else:
            g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.run_to_completion(tol=TOL, check_every=CHECK)
        return g.tallies().f


def features(cfgs, dt, period_steps):
    """Network inputs: the configured values, with the pulse period actually
    simulated."""
    return np.stack([synth.surrogate_features(c, float(p) * float(d) if c["pulses"] > 1 else 0.0)
                     for c, d, p in zip(cfgs, dt, period_steps)])


class Surrogate:
    """An ensemble of networks for f (it_mlp_*).

    Fall-back gate: an answer is accepted when the ensemble's spread (max -
    min over the members) is at most tau.  tau is at most the spread limit
    (1e-3), so every answer whose spread exceeds the limit falls back; with a
    held-out slice of the training runs it is lowered to the largest spread at
    which the accepted held-out answers are within `tol` of the solver at the
    rate `coverage` -- members trained on few runs can agree on a biased
    answer, and their spread then understates the error."""

    def __init__(self, members=5, max_batch=1024, seed=1610067495):
        self.members = members
        self.h = B.it_mlp_create(members, max_batch)
        self.tau = None          # None: the spread limit itself
        theta = synth.mlp_init(seed, members)
        for m in range(members):
            B.it_mlp_set_params(self.h, m, theta[m])

    def fit(self, X, y, epochs=200, batch=256, lr=1e-3, seed=1, lr_min=None, chunks=20, val_frac=0.0,
            coverage=0.99, tol=1e-3, spread_max=1e-3, split_seed=1610067496):
        """Adam over the training set; with lr_min the rate follows a cosine
        from lr down to lr_min in `chunks` steps of epochs/chunks epochs.
        With val_frac > 0 a seeded random slice of that fraction is held out
        of training and calibrates tau (see the class)."""
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        nval = int(round(val_frac * len(y)))
        if nval > 0:
            order = np.argsort(synth.uniform01(split_seed, len(y)), kind="stable")
            val, trn = order[:nval], order[nval:]
            Xv, yv, X, y = X[val], y[val], X[trn], y[trn]
        B.it_mlp_fit_normalization(self.h, X)
        B.it_mlp_set_data(self.h, X, y)
        if lr_min is None:
            loss = B.it_mlp_train(self.h, epochs, batch, lr, seed)
        else:
            losses = []
            per = max(1, epochs // chunks)
            for c in range(chunks):
                r = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * c / chunks))
                losses.append(B.it_mlp_train(self.h, per, batch, r, seed + c))
            loss = np.concatenate(losses)
        if nval > 0:
            self.calibrate(Xv, yv, coverage, tol, spread_max)
        return loss

    def calibrate(self, X, y, coverage=0.99, tol=1e-3, spread_max=1e-3, confidence=0.95):
        """tau = the largest held-out spread s <= spread_max such that, of the
        held-out answers with spread <= s, the fraction within tol of y is at
        least `coverage` with one-sided confidence `confidence`: the
        Clopper-Pearson lower bound of that binomial proportion (the
        (1 - confidence) quantile of Beta(k, n - k + 1) for k of n within
        tol) must reach `coverage`.  With every accepted answer within tol
        this needs n >= ln(1 - confidence) / ln(coverage) answers (298 for
        0.99 at 95 %).  0 (every answer falls back) when no such s exists.
        (X, y) must not be training data."""
        from scipy.stats import beta
        mean, spread = self.predict(X)
        ok = np.abs(mean - np.asarray(y)) <= tol
        order = np.argsort(spread, kind="stable")
        s_sorted, ok_sorted = spread[order], ok[order]
        good = np.cumsum(ok_sorted)
        tau = 0.0
        for k in range(len(order)):
            if s_sorted[k] > spread_max:
                break
            # accept up to and including the last answer with this spread
            if k + 1 < len(order) and s_sorted[k + 1] == s_sorted[k]:
                continue
            n, g = k + 1, int(good[k])
            lower = float(beta.ppf(1.0 - confidence, g, n - g + 1)) if g > 0 else 0.0
            if lower >= coverage:
                tau = float(s_sorted[k])
        self.tau = tau
        return tau

    def gate(self, spread_max=1e-3):
        """The spread up to which answers are accepted."""
        return spread_max if self.tau is None else min(spread_max, self.tau)

    def predict(self, X):
        mean, spread, _ = B.it_mlp_predict(self.h, self.members, X)
        return mean, spread

    def close(self):
        if getattr(self, "h", None):
            B.it_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def answer(sur: Surrogate, cfgs, dt, period_steps, spread_max=1e-3, batched=False):
    """f for each configuration: the ensemble mean where the spread is within
    the calibrated gate (at most spread_max), else the solver -- one context
    per configuration, or with batched=True all fall-backs in one batch (the
    same per-cell arithmetic, so the same f to summation order).  Returns (f,
    used_solver mask, seconds)."""
    t0 = time.perf_counter()
    X = features(cfgs, dt, period_steps)
    mean, spread = sur.predict(X)
    f = mean.copy()
    fb = spread > sur.gate(spread_max)
    idx = np.nonzero(fb)[0]
    if batched and len(idx):
        f[idx] = solve_batch([cfgs[i] for i in idx])[0]
    else:
        for i in idx:
            f[i] = solve_plain(cfgs[i], dt[i], period_steps[i])
    return f, fb, time.perf_counter() - t0


def main(argv=None, quiet=False):
    """Generate solver data, train the ensemble, answer held-out
    configurations with fall-back, and compare with the plain solver.
    Returns the summary (and prints it as one JSON line unless quiet)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-min", type=float, default=1e-5)
    ap.add_argument("--members", type=int, default=5)
    ap.add_argument("--plain-sample", type=int, default=200)
    ap.add_argument("--spread", type=float, default=1e-3)
    ap.add_argument("--val-frac", type=float, default=0.1, help="training runs held out to calibrate the gate")
    ap.add_argument("--coverage", type=float, default=0.99)
    ap.add_argument("--single-pulse", action="store_true",
                    help="keep only the single-pulse configurations of the --train / --test draws")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    tr_cfg = synth.surrogate_configs(1610067493, a.train)
    te_cfg = synth.surrogate_configs(1610067494, a.test)
    if a.single_pulse:
        tr_cfg = [c for c in tr_cfg if c["pulses"] == 1]
        te_cfg = [c for c in te_cfg if c["pulses"] == 1]
    a.train, a.test = len(tr_cfg), len(te_cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f_tr, dt_tr, p_tr = solve_batch(tr_cfg)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    f_te, dt_te, p_te = solve_batch(te_cfg)
    t_te_batch = time.perf_counter() - t0
    X_tr, X_te = features(tr_cfg, dt_tr, p_tr), features(te_cfg, dt_te, p_te)
    sur = Surrogate(members=a.members)
    t0 = time.perf_counter()
    loss = sur.fit(X_tr, f_tr, epochs=a.epochs, lr=a.lr, lr_min=a.lr_min, val_frac=a.val_frac,
                   coverage=a.coverage, tol=1e-3, spread_max=a.spread)
    t_fit = time.perf_counter() - t0
    t0 = time.perf_counter()
    mean, spread = sur.predict(X_te)
    t_pred = time.perf_counter() - t0
    err = np.abs(mean - f_te)
    acc = spread <= sur.gate(a.spread)
    # answers with fall-back to the solver: all held-out configurations with the
    # fall-backs in one batch; with one context per fall-back on the plain sample
    k = min(a.plain_sample, a.test)
    f_ansb, fb, t_ansb = answer(sur, te_cfg, dt_te, p_te, a.spread, batched=True)
    f_ans, _, t_ans = answer(sur, te_cfg[:k], dt_te[:k], p_te[:k], a.spread)
    # the plain solver alone, timed on the same sample
    t0 = time.perf_counter()
    f_pl = np.array([solve_plain(c, d, p) for c, d, p in zip(te_cfg[:k], dt_te[:k], p_te[:k])])
    t_pl = time.perf_counter() - t0
    acc_ok = float(np.mean(err[acc] <= 1e-3)) if acc.any() else None
    within = acc_ok is not None and acc_ok >= a.coverage
    out = {
        "train": a.train, "test": a.test, "single_pulse": a.single_pulse, "members": a.members, "epochs": a.epochs,
        "val_frac": a.val_frac, "coverage": a.coverage, "gate_spread": sur.gate(a.spread),
        "data_gen_s": t_gen, "data_gen_solves_per_s": a.train / t_gen,
        "fit_s": t_fit, "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
        "test_err_median": float(np.median(err)), "test_err_p90": float(np.quantile(err, 0.9)),
        "test_err_max": float(err.max()),
        "accepted_fraction": float(acc.mean()),
        "accepted_err_le_1e3": acc_ok,
        "accepted_within_coverage": within,
        "answer_err_max": float(np.max(np.abs(f_ansb - f_te))),
        "answer_err_le_1e3": float(np.mean(np.abs(f_ansb - f_te) <= 1e-3)),
        "fallback_fraction": float(fb.mean()),
        "predict_only_solves_per_s": a.test / t_pred,
        "surrogate_with_fallback_solves_per_s": k / t_ans,
        "surrogate_with_batched_fallback_solves_per_s": a.test / t_ansb,
        "plain_fallback_answer_err_max": float(np.max(np.abs(f_ans - f_te[:k]))),
        "plain_solves_per_s": k / t_pl,
        "batched_solves_per_s": a.test / t_te_batch,
        # a gain is reported only while the accepted answers meet the coverage
        "gain_vs_batched": (a.test / t_ansb) / (a.test / t_te_batch) if within else None,
        "gain_vs_plain": (a.test / t_ansb) / (k / t_pl) if within else None,
        "plain_vs_batch_max_abs_df": float(np.max(np.abs(f_pl - f_te[:k]))),
    }
    sur.close()
    if not quiet:
        print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
