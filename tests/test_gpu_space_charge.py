"""Parity of the optional space-charge term with the FP64 oracle.

With the term on, each species' update also carries -/+ mu n div E, where
div E = q/eps0 (n+ - n-) (Maxwell-Gauss, Eq. theEquation), evaluated on the
old level like the recombination sink.  On these cases the term moves the
densities by 30-80 % of their maximum and adds a tally of 1-10 % of the
released charge, so a wrong sign, species or level fails the 1e-4 bound by
orders of magnitude.  The tolerances are those of the term-free parity
tests: densities 1e-4 of the maximum (FP32 storage) or 1e-12 (FP64), f
within 1e-5, charges within 1e-5 of the released total.
"""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu

MU, DD, ALPHA = (1.73, 1.87), (0.037, 0.037), 1.6e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()


def _scheme(s):
    return o.SCHEME_UPWIND if s == B.IT_UPWIND else o.SCHEME_LAX_WENDROFF


def _dt(dx, V, nz, tr, scheme=B.IT_LAX_WENDROFF):
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm) if len(tr) else 0.0
    return o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, scheme=_scheme(scheme), space_charge=True)


def _pair(nx, ny, nz, dx, V, dt, lateral=B.IT_PERIODIC, scheme=B.IT_LAX_WENDROFF, kernel=B.IT_KERNEL_AUTO,
          precision=B.IT_FP32):
    g = B.Simulation(nx, ny, nz, dx, V, dt_s=dt, precision=precision, lateral_bc=lateral, scheme=scheme,
                     kernel=kernel, space_charge=True)
    O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V,
                 lateral_bc=o.LATERAL_ABSORBING if lateral == B.IT_ABSORBING else o.LATERAL_PERIODIC,
                 scheme=_scheme(scheme), space_charge=True)
    return g, O


def _close(gpu, orc, tol, what=""):
    scale = np.max(np.abs(orc))
    err = np.max(np.abs(gpu.astype(np.float64) - orc)) / scale
    assert err <= tol, f"{what}: max abs error / max = {err:.3e} > {tol}"


def _tallies(tg, to, f_tol, rel_tol):
    assert tg.f == pytest.approx(to.f, abs=f_tol)
    tot = to.released.sum()
    np.testing.assert_allclose(tg.released, to.released, rtol=rel_tol)
    for name in ("in_domain", "collected_anode", "collected_cathode", "lost_lateral", "space_charge"):
        np.testing.assert_allclose(getattr(tg, name), getattr(to, name), rtol=0, atol=rel_tol * tot,
                                   err_msg=name)
    assert tg.recombined == pytest.approx(to.recombined, abs=rel_tol * tot)
    # the term is exercised: its tally is far above the comparison's bound
    assert np.all(np.abs(to.space_charge) > 100 * rel_tol * tot)


SC_CASES = [
    # nx, ny, nz, dx, V, lateral, scheme, kernel, n_tracks
    (36, 20, 23, 5e-4, 200.0, B.IT_ABSORBING, B.IT_LAX_WENDROFF, B.IT_KERNEL_ZMARCH, 7),
    (64, 48, 40, 4e-4, 100.0, B.IT_PERIODIC, B.IT_LAX_WENDROFF, B.IT_KERNEL_ZMARCH, 25),
    (64, 48, 40, 4e-4, 100.0, B.IT_ABSORBING, B.IT_UPWIND, B.IT_KERNEL_ZMARCH, 25),
    (256, 16, 12, 5e-4, 300.0, B.IT_PERIODIC, B.IT_LAX_WENDROFF, B.IT_KERNEL_ZMARCH2, 40),
    (512, 8, 10, 5e-4, 300.0, B.IT_ABSORBING, B.IT_LAX_WENDROFF, B.IT_KERNEL_ZMARCH2, 40),
    (64, 48, 40, 4e-4, 100.0, B.IT_ABSORBING, B.IT_UPWIND, B.IT_KERNEL_ZMARCH2, 25),
    (37, 19, 13, 5e-4, 200.0, B.IT_PERIODIC, B.IT_LAX_WENDROFF, B.IT_KERNEL_SIMPLE, 6),
    (37, 19, 13, 5e-4, 200.0, B.IT_ABSORBING, B.IT_UPWIND, B.IT_KERNEL_SIMPLE, 6),
]


@pytest.mark.parametrize("case", SC_CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-bc{c[5]}-s{c[6]}-k{c[7]}")
def test_small_grids_with_space_charge_match_oracle(case):
    nx, ny, nz, dx, V, lat, sch, ker, nt = case
    tr = synth.uniform_tracks(100 + nx + ny, nt, nx * dx, ny * dx, 1e-3, let="loguniform")
    tr.x_cm[0] = 0.2 * dx
    tr.y_cm[0] = (ny - 0.3) * dx
    g, O = _pair(nx, ny, nz, dx, V, _dt(dx, V, nz, tr, sch), lateral=lat, scheme=sch, kernel=ker)
    with g:
        assert g.launch()["kernel"] == ker
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        done = 0
        for chk in (1, 7, 40, 75):
            g.step(chk - done)
            O.step(chk - done)
            done = chk
            for s in range(2):
                _close(g.density(s), O.density(s), 1e-4, what=f"step {chk} species {s}")
        _tallies(g.tallies(), O.tallies(), 1e-5, 1e-5)


@pytest.mark.parametrize("lat", [B.IT_PERIODIC, B.IT_ABSORBING])
def test_space_charge_fp64_storage_matches_oracle_to_rounding(lat):
    nx, ny, nz, dx, V = 24, 20, 30, 5e-4, 150.0
    tr = synth.uniform_tracks(9, 5, nx * dx, ny * dx, 1e-3)
    g, O = _pair(nx, ny, nz, dx, V, _dt(dx, V, nz, tr), lateral=lat, precision=B.IT_FP64)
    with g:
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.step(60)
        O.step(60)
        for s in range(2):
            _close(g.density(s), O.density(s), 1e-12, what=f"species {s}")
        tg, to = g.tallies(), O.tallies()
        assert tg.f == pytest.approx(to.f, abs=1e-12)
        np.testing.assert_allclose(tg.space_charge, to.space_charge, rtol=1e-10)


def test_space_charge_kernels_agree_bitwise_and_balance_the_charge():
    # the term is one more operation after upd7 in every kernel, in the same
    # order, so every kernel and launch shape still agrees bitwise; with its
    # tally the charge balance released + space_charge = in_domain +
    # collected + lost_lateral + recombined closes
    nx, ny, nz, dx, V = 64, 32, 24, 5e-4, 200.0
    tr = synth.uniform_tracks(4, 10, nx * dx, ny * dx, 1e-3)
    dt = _dt(dx, V, nz, tr)
    shapes = [(B.IT_KERNEL_SIMPLE, 0, 0, 0, 0), (B.IT_KERNEL_ZMARCH, 0, 0, 0, 0),
              (B.IT_KERNEL_ZMARCH, 4, 2, 3, -1), (B.IT_KERNEL_ZMARCH, 16, 1, 5, 7),
              (B.IT_KERNEL_ZMARCH2, 0, 0, 0, 0), (B.IT_KERNEL_ZMARCH2, 32, 1, 3, -1),
              (B.IT_KERNEL_ZMARCH2, 16, 2, 6, 5)]
    out = []
    for lat in (B.IT_PERIODIC, B.IT_ABSORBING):
        for ker, ty, cps, S, grid in shapes:
            with B.Simulation(nx, ny, nz, dx, V, dt_s=dt, lateral_bc=lat, space_charge=True) as g:
                g.set_launch(ker, ty, cps, S, grid)
                g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
                g.step(51)
                t = g.tallies()
                assert np.all(t.space_charge < 0)
                for s in range(2):
                    lhs = t.released[s] + t.space_charge[s]
                    rhs = t.in_domain[s] + t.collected[s] + t.lost_lateral[s] + t.recombined
                    assert rhs == pytest.approx(lhs, rel=2e-6), (lat, ker, s)
                out.append((lat, g.density(0), g.density(1), t))
    for lat in (B.IT_PERIODIC, B.IT_ABSORBING):
        runs = [r for r in out if r[0] == lat]
        for _, d0, d1, t in runs[1:]:
            assert np.array_equal(d0, runs[0][1]) and np.array_equal(d1, runs[0][2])
            assert t.f == pytest.approx(runs[0][3].f, abs=1e-8)
            np.testing.assert_allclose(t.space_charge, runs[0][3].space_charge, rtol=1e-6)


@pytest.mark.parametrize("bc", [B.IT_PERIODIC, B.IT_ABSORBING])
def test_space_charge_batch_equals_single_contexts_bitwise(bc):
    # nx a multiple of 4 (float4 kernel) and not (scalar kernel), one plane
    shapes = [(32, 32, 32, 4e-4, 120.0), (37, 20, 23, 5e-4, 300.0), (16, 16, 1, 5e-4, 200.0),
              (40, 12, 60, 6e-4, 400.0)]
    cases = []
    for q, (nx, ny, nz, dx, V) in enumerate(shapes):
        tr = synth.uniform_tracks(700 + q, 3 + 2 * q, nx * dx, ny * dx, 8e-4, let="loguniform")
        npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
        cases.append((dict(nx=nx, ny=ny, nz=nz, dx_cm=dx, voltage_V=V, n_peak_cm3=npk), tr))
    steps = 40
    with B.Batch([d for d, _ in cases], lateral_bc=bc, space_charge=True) as bt:
        bt.set_chunk(1024)
        for q, (_, tr) in enumerate(cases):
            bt.deposit(q, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.run(tol=0.0, max_steps=steps, check_every=8)
        for q, (d, tr) in enumerate(cases):
            tb = bt.tallies(q)
            with B.Simulation(d["nx"], d["ny"], d["nz"], d["dx_cm"], d["voltage_V"],
                              n_peak_cm3=d["n_peak_cm3"], lateral_bc=bc, space_charge=True) as g:
                g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
                g.step(steps)
                ts = g.tallies()
                assert ts.dt_s == tb.dt_s
                # the automatic dt honours the space-charge bound
                assert ts.dt_s == pytest.approx(o.dt_rule(d["dx_cm"], d["voltage_V"], d["nz"] * d["dx_cm"],
                                                          n_peak=d["n_peak_cm3"], space_charge=True), rel=1e-14)
                for s in range(2):
                    assert np.array_equal(bt.density(q, s), g.density(s)), f"sim {q} species {s}"
                assert tb.f == pytest.approx(ts.f, abs=1e-7)
                np.testing.assert_allclose(tb.space_charge, ts.space_charge, rtol=1e-6)


def test_space_charge_full_size_in_the_autotuned_launch_shape():
    # the 256 x 256 x 400 pulsed workload with the term on, in the launch
    # shape the autotuner picks, against the oracle after 4 steps
    w = synth.pulsed_256x256x400(200.0)
    tr = synth.pulsed_tracks(w)
    g, O = _pair(w.nx, w.ny, w.nz, w.dx_cm, w.voltage_V, _dt(w.dx_cm, w.voltage_V, w.nz, tr))
    with g:
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.autotune(trial_steps=4, force=True)
        assert g.launch()["kernel"] in (B.IT_KERNEL_ZMARCH, B.IT_KERNEL_ZMARCH2)
        g.step(4)
        O.step(4)
        for s in range(2):
            _close(g.density(s), O.density(s), 1e-4, what=f"species {s}")
        tg, to = g.tallies(), O.tallies()
        assert tg.f == pytest.approx(to.f, abs=1e-5)
        tot = to.released.sum()
        np.testing.assert_allclose(tg.space_charge, to.space_charge, rtol=0, atol=1e-5 * tot)
