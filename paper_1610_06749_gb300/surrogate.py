"""Surrogate workflow: solver-generated data, ensemble training, prediction
with a fall-back to the solver.

Orchestration only -- every solve runs in the CUDA solver (batched or one
context per configuration), every training and inference step in the CUDA
network kernels; this module moves arrays between them.

A configuration (synth.surrogate_configs) is released as one pulse, or a
train of 4 identical pulses; its time step is the automatic rule with the
recombination bound taken from the deposited pulse's peak times the pulse
count, and a train's period is rounded to a whole number of 64-step check
intervals (the period actually simulated is the sixth network input).  Runs
to completion use the upwind drift (stable at the recombination-bound time
step, where Lax-Wendroff diverges).
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B
from . import synth

CHECK = synth.SURROGATE_CHECK
TOL = 1e-6


def _desc(c):
    return dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], dx_cm=c["dx_cm"], voltage_V=c["voltage_V"])


def solve_batch(cfgs, chunk=2048):
    """f of every configuration with the batched solver.  Returns (f, dt,
    period_steps) arrays."""
    n = len(cfgs)
    f = np.full(n, np.nan)
    dt = np.zeros(n)
    per = np.zeros(n, dtype=np.int64)
    for a in range(0, n, chunk):
        part = cfgs[a:a + chunk]
        with B.Batch([_desc(c) for c in part], scheme=B.IT_UPWIND) as bt:
            for k, c in enumerate(part):
                tr = synth.surrogate_tracks(c)
                bt.deposit(k, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
                if c["pulses"] > 1:
                    bt.set_pulses(k, c["pulses"], CHECK)      # provisional period: the count sets the dt bound
            bt.retime()
            for k, c in enumerate(part):
                dt[a + k] = bt.tallies(k).dt_s
                if c["pulses"] > 1:
                    p = max(1, int(round(c["period_s"] / dt[a + k] / CHECK))) * CHECK
                    per[a + k] = p
                    bt.set_pulses(k, c["pulses"], p)
            bt.run(tol=TOL, check_every=CHECK)
            for k in range(len(part)):
                f[a + k] = bt.tallies(k).f
    return f, dt, per


def solve_plain(c, dt, period_steps):
    """f of one configuration with one solver context (the method without the
    surrogate), at the given time step and pulse period."""
    with B.Simulation(c["nx"], c["ny"], c["nz"], c["dx_cm"], c["voltage_V"], dt_s=dt,
                      scheme=B.IT_UPWIND) as g:
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

    def calibrate(self, X, y, coverage=0.99, tol=1e-3, spread_max=1e-3, min_accept=10):
        """tau = the largest held-out spread s <= spread_max such that, of the
        held-out answers with spread <= s (at least min_accept of them), the
        fraction within tol of y is >= coverage; 0 (every answer falls back)
        when no such s exists.  (X, y) must not be training data."""
        mean, spread = self.predict(X)
        ok = np.abs(mean - np.asarray(y)) <= tol
        order = np.argsort(spread, kind="stable")
        s_sorted, ok_sorted = spread[order], ok[order]
        good = np.cumsum(ok_sorted)
        n = np.arange(1, len(order) + 1)
        tau = 0.0
        for k in range(len(order)):
            if s_sorted[k] > spread_max:
                break
            # accept up to and including the last answer with this spread
            if k + 1 < len(order) and s_sorted[k + 1] == s_sorted[k]:
                continue
            if n[k] >= min_accept and good[k] >= coverage * n[k]:
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
    a = ap.parse_args(argv)
    from . import build
    build.build()
    tr_cfg = synth.surrogate_configs(1610067493, a.train)
    te_cfg = synth.surrogate_configs(1610067494, a.test)
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
    # answers with fall-back to the solver (all held-out configurations)
    f_ans, fb, t_ans = answer(sur, te_cfg, dt_te, p_te, a.spread)
    f_ansb, _, t_ansb = answer(sur, te_cfg, dt_te, p_te, a.spread, batched=True)
    # the plain solver alone, timed on a sample
    k = min(a.plain_sample, a.test)
    t0 = time.perf_counter()
    f_pl = np.array([solve_plain(c, d, p) for c, d, p in zip(te_cfg[:k], dt_te[:k], p_te[:k])])
    t_pl = time.perf_counter() - t0
    out = {
        "train": a.train, "test": a.test, "members": a.members, "epochs": a.epochs,
        "val_frac": a.val_frac, "coverage": a.coverage, "gate_spread": sur.gate(a.spread),
        "data_gen_s": t_gen, "data_gen_solves_per_s": a.train / t_gen,
        "fit_s": t_fit, "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
        "test_err_median": float(np.median(err)), "test_err_p90": float(np.quantile(err, 0.9)),
        "test_err_max": float(err.max()),
        "accepted_fraction": float(acc.mean()),
        "accepted_err_le_1e3": float(np.mean(err[acc] <= 1e-3)) if acc.any() else None,
        "answer_err_max": float(np.max(np.abs(f_ans - f_te))),
        "answer_err_le_1e3": float(np.mean(np.abs(f_ans - f_te) <= 1e-3)),
        "fallback_fraction": float(fb.mean()),
        "predict_only_solves_per_s": a.test / t_pred,
        "surrogate_with_fallback_solves_per_s": a.test / t_ans,
        "surrogate_with_batched_fallback_solves_per_s": a.test / t_ansb,
        "batched_fallback_answer_err_max": float(np.max(np.abs(f_ansb - f_te))),
        "plain_solves_per_s": k / t_pl,
        "batched_solves_per_s": a.test / t_te_batch,
        "plain_vs_batch_max_abs_df": float(np.max(np.abs(f_pl - f_te[:k]))),
    }
    sur.close()
    if not quiet:
        print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
