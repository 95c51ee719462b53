"""Batched simulations: each simulation in a batch computes what a single
context with the same parameters computes (bitwise-identical densities, f to
FP64 summation order), and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()


def small_descs():
    # uneven grids, including nx not a multiple of 4 and a single plane
    shapes = [(32, 32, 32, 4e-4, 120.0), (37, 20, 23, 5e-4, 300.0), (64, 48, 40, 3e-4, 50.0),
              (16, 16, 1, 5e-4, 200.0), (40, 12, 60, 6e-4, 400.0), (24, 24, 24, 2e-4, 80.0)]
    out = []
    for q, (nx, ny, nz, dx, V) in enumerate(shapes):
        tr = synth.uniform_tracks(500 + q, 3 + 2 * q, nx * dx, ny * dx, 8e-4, let="loguniform")
        npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
        out.append((dict(nx=nx, ny=ny, nz=nz, dx_cm=dx, voltage_V=V, n_peak_cm3=npk), tr))
    return out


@pytest.mark.parametrize("bc", [B.IT_PERIODIC, B.IT_ABSORBING])
def test_batch_equals_single_contexts_bitwise(bc):
    cases = small_descs()
    steps = 40
    with B.Batch([d for d, _ in cases], lateral_bc=bc) as bt:
        bt.set_chunk(1024)           # several entries per simulation
        for q, (_, tr) in enumerate(cases):
            bt.deposit(q, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.run(tol=0.0, max_steps=steps, check_every=8)
        for q, (d, tr) in enumerate(cases):
            tb = bt.tallies(q)
            assert tb.steps == steps
            with B.Simulation(d["nx"], d["ny"], d["nz"], d["dx_cm"], d["voltage_V"],
                              n_peak_cm3=d["n_peak_cm3"], lateral_bc=bc) as g:
                g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
                g.step(steps)
                ts = g.tallies()
                assert ts.dt_s == tb.dt_s
                for s in range(2):
                    assert np.array_equal(bt.density(q, s), g.density(s)), f"sim {q} species {s}"
                # the single context may run the z-march kernel, whose tally
                # partials are FP32 over up to 32 planes before FP64
                assert tb.f == pytest.approx(ts.f, abs=1e-7)
                # in-domain sums: FP32 partials over 32 cells, grouped differently
                np.testing.assert_allclose(tb.in_domain, ts.in_domain, rtol=1e-8)
                np.testing.assert_allclose(tb.released, ts.released, rtol=1e-15)


def test_batch_autotune_keeps_the_state_and_changes_only_the_work_split():
    cases = small_descs()
    steps = 24
    runs = []
    for tune in (False, True):
        with B.Batch([d for d, _ in cases]) as bt:
            for q, (_, tr) in enumerate(cases):
                bt.deposit(q, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
            before = [bt.tallies(q) for q in range(len(cases))]
            if tune:
                us = bt.autotune(trial_steps=4)
                assert np.isfinite(us) and us > 0
                after = [bt.tallies(q) for q in range(len(cases))]
                for t0, t1 in zip(before, after):   # trial steps leave no trace
                    assert t1.steps == 0 and t1.recombined == 0.0
                    np.testing.assert_array_equal(t1.in_domain, t0.in_domain)
            bt.run(tol=0.0, max_steps=steps, check_every=8)
            if tune:
                with pytest.raises(B.ItError):
                    bt.autotune()            # only before the first step
            runs.append(([bt.density(q, 0) for q in range(len(cases))],
                         [bt.tallies(q) for q in range(len(cases))]))
    (d0, t0), (d1, t1) = runs
    for q in range(len(cases)):
        assert np.array_equal(d0[q], d1[q]), f"sim {q}"
        assert t1[q].steps == t0[q].steps == steps
        assert t1[q].f == pytest.approx(t0[q].f, abs=1e-12)


def test_batch_runs_to_completion_and_matches_oracle():
    cases = small_descs()[:3]
    with B.Batch([d for d, _ in cases]) as bt:
        for q, (_, tr) in enumerate(cases):
            bt.deposit(q, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.run(tol=1e-7, check_every=16)
        for q, (d, tr) in enumerate(cases):
            tb = bt.tallies(q)
            assert tb.in_domain.sum() / tb.released.sum() < 1e-7
            O = o.Oracle(d["nx"], d["ny"], d["nz"], d["dx_cm"], tb.dt_s, voltage_V=d["voltage_V"])
            O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
            O.step(tb.steps)
            to = O.tallies()
            assert tb.f == pytest.approx(to.f, abs=1e-5)
            for s in range(2):
                tot = tb.in_domain[s] + tb.collected[s] + tb.lost_lateral[s] + tb.recombined
                assert tot == pytest.approx(tb.released[s], rel=2e-6)


def test_batch_rejects_bad_input_and_skips_empty_simulations():
    d = dict(nx=8, ny=8, nz=8, dx_cm=5e-4, voltage_V=100.0)
    with pytest.raises(B.ItError) as e:
        B.Batch([d, dict(d, nx=0)])
    assert e.value.code == B.IT_EINVAL and "simulation 1" in str(e.value)
    with B.Batch([d, d]) as bt:
        bt.deposit(0, [2e-3], [2e-3], [5.0], [1e-3])
        bt.run(tol=1e-6, check_every=4)
        assert bt.tallies(1).steps == 0 and bt.tallies(1).released.sum() == 0.0
        assert bt.tallies(0).steps > 0
        with pytest.raises(B.ItError) as e:
            bt.deposit(1, [2e-3], [2e-3], [5.0], [1e-3])
        assert e.value.code == B.IT_ESTATE


def test_full_occupancy_runner_keeps_every_simulation_active():
    # the runner behind the batched kernel's profile: the first 8 simulations
    # of the batched workload, autotuned, 64 steps with all of them active
    from paper_1610_06749_gb300 import batched
    r = batched.full_occupancy(n_sims=8, steps=64)
    assert r["sims"] == 8 and r["steps"] == 64 and r["sims_active_throughout"] == 8
    assert r["autotuned_us_per_step"] > 0 and r["run_us_per_step"] > 0
    assert r["cells"] == sum(d["nx"] * d["ny"] * d["nz"] for d in synth.batch_descriptors()[:8])
