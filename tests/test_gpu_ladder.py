"""The doubling dt ladder of it_run_to_completion against the oracle's.

Both sides decide each rung themselves from their own state's peak density
(the oracle in FP64, the library from the exact maximum of its FP32 field),
so the decisions are compared, not replayed: the logs must agree step for
step and dt for dt.  A rung flips only if the peak density lies within the
densities' parity error (1e-4) of a power-of-two threshold, which these
seeded cases do not come near (the test reports the margin).  Densities and
tallies then meet the bounds of the fixed-step parity tests.
"""
import math

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


def dense_pulse(seed=11):
    # six tracks of 100-720 keV/um on a 24 x 24 x 40 grid at 50 V
    nx, ny, nz, dx, V = 24, 24, 40, 5e-4, 50.0
    tr = synth.uniform_tracks(seed, 6, nx * dx, ny * dx, 1e-3, let="loguniform")
    tr.let_keV_um[:] = np.maximum(tr.let_keV_um, 100.0)
    return nx, ny, nz, dx, V, tr


def _oscheme(s):
    return o.SCHEME_UPWIND if s == B.IT_UPWIND else o.SCHEME_LAX_WENDROFF


def _margin(log, kappa=0.5):
    """Smallest relative distance of a deciding peak density from the rung
    thresholds kappa / (alpha dt 2^j) next to it."""
    m = math.inf
    for _, dt, nmax in log[1:]:
        for r in (dt, 2.0 * dt):
            m = min(m, abs(nmax - kappa / (ALPHA * r)) / nmax)
    return m


@pytest.mark.parametrize("scheme", [B.IT_UPWIND, B.IT_LAX_WENDROFF])
@pytest.mark.parametrize("kernel", [B.IT_KERNEL_ZMARCH, B.IT_KERNEL_SIMPLE])
def test_ladder_matches_the_oracle_ladder(scheme, kernel):
    nx, ny, nz, dx, V, tr = dense_pulse()
    npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
    dt0 = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk, scheme=_oscheme(scheme))
    O = o.Oracle(nx, ny, nz, dx, dt0, mu=MU, D=DD, alpha=ALPHA, voltage_V=V, scheme=_oscheme(scheme))
    O.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
    with B.Simulation(nx, ny, nz, dx, V, dt_s=dt0, scheme=scheme, kernel=kernel, dt_ladder=True) as g:
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        # three checks (steps 0, 64, 128), then stop at 160 on both sides
        with pytest.raises(B.ItError) as e:
            g.run_to_completion(tol=1e-6, max_steps=160, check_every=64)
        assert e.value.code == B.IT_ETIMEOUT
        steps, done, olog = O.run_to_completion(1e-6, 160, 64, ladder=True)
        assert steps == 160 and not done
        glog = g.dt_log()
        assert _margin(olog) > 1e-3
        assert [(s, dt) for s, dt, _ in glog] == [(s, dt) for s, dt, _ in olog]
        assert len(glog) >= 3                      # the ladder did rise
        for (_, _, a), (_, _, b) in zip(glog[1:], olog[1:]):
            assert a == pytest.approx(b, rel=1e-4)
        tg, to = g.tallies(), O.tallies()
        assert tg.steps == to.steps == 160
        assert tg.t_s == pytest.approx(to.t_s, rel=1e-14)
        for s in range(2):
            d, w = g.density(s), O.density(s)
            assert np.max(np.abs(d - w)) <= 1e-4 * np.max(np.abs(w))
        assert tg.f == pytest.approx(to.f, abs=1e-5)
        tot = to.released.sum()
        assert tg.recombined == pytest.approx(to.recombined, abs=1e-5 * tot)
        # on to completion: the same number of steps and f
        n_more = g.run_to_completion(tol=1e-6, max_steps=100_000, check_every=64)
        steps2, done2, _ = O.run_to_completion(1e-6, 100_000, 64, ladder=True)
        assert done2 and n_more == steps2
        assert g.tallies().f == pytest.approx(O.tallies().f, abs=1e-5)


@pytest.mark.parametrize("bc", [B.IT_PERIODIC, B.IT_ABSORBING])
def test_ladder_batch_equals_single_contexts_bitwise(bc):
    # the batch applies the same rungs per simulation, so each simulation
    # takes the same steps as in its own context and agrees bitwise
    shapes = [(24, 24, 40, 5e-4, 50.0), (32, 20, 30, 4e-4, 120.0), (37, 21, 25, 6e-4, 300.0),
              (16, 16, 1, 5e-4, 200.0)]
    cases = []
    for q, (nx, ny, nz, dx, V) in enumerate(shapes):
        tr = synth.uniform_tracks(900 + q, 4 + q, nx * dx, ny * dx, 1e-3, let="loguniform")
        tr.let_keV_um[:] = np.maximum(tr.let_keV_um, 50.0)
        npk = o.peak_track_density(tr.let_keV_um, tr.b_cm)
        cases.append((dict(nx=nx, ny=ny, nz=nz, dx_cm=dx, voltage_V=V, n_peak_cm3=npk), tr))
    steps = 256
    with B.Batch([d for d, _ in cases], lateral_bc=bc, scheme=B.IT_UPWIND, dt_ladder=True) as bt:
        for q, (_, tr) in enumerate(cases):
            bt.deposit(q, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.run(tol=0.0, max_steps=steps, check_every=64)
        for q, (d, tr) in enumerate(cases):
            tb = bt.tallies(q)
            with B.Simulation(d["nx"], d["ny"], d["nz"], d["dx_cm"], d["voltage_V"], n_peak_cm3=d["n_peak_cm3"],
                              lateral_bc=bc, scheme=B.IT_UPWIND, dt_ladder=True) as g:
                g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
                with pytest.raises(B.ItError):
                    g.run_to_completion(tol=0.0, max_steps=steps, check_every=64)
                ts = g.tallies()
                assert ts.steps == tb.steps == steps
                assert ts.dt_s == tb.dt_s
                assert ts.t_s == pytest.approx(tb.t_s, rel=1e-14)   # the sum grouped by segment
                if q == 0:   # 50 V, dense: the reaction bound starts far below the Eq. (vNeum) step
                    assert len(g.dt_log()) >= 2, "the ladder never rose"
                for s in range(2):
                    assert np.array_equal(bt.density(q, s), g.density(s)), f"sim {q} species {s}"
                assert tb.f == pytest.approx(ts.f, abs=1e-7)


def test_ladder_batch_pulse_train_equals_single_context_bitwise():
    # a train of 4 pulses: the ladder applies only once the last pulse is in;
    # the batch's check at the step of the last pulse, which runs after that
    # pulse's deposit, counts it as still to come exactly like a context,
    # whose check runs before the deposits of its step
    nx, ny, nz, dx, V, P = 32, 32, 30, 5e-4, 150.0, 128
    tr = synth.uniform_tracks(931, 9, nx * dx, ny * dx, 1e-3, let="loguniform")
    tr.let_keV_um[:] = np.maximum(tr.let_keV_um, 50.0)
    d = dict(nx=nx, ny=ny, nz=nz, dx_cm=dx, voltage_V=V)
    with B.Batch([d], scheme=B.IT_UPWIND, dt_ladder=True, react_kappa=0.0625) as bt:
        bt.deposit(0, tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        bt.set_pulses(0, 4, P)
        bt.retime()
        dt0 = bt.tallies(0).dt_s
        bt.run(tol=1e-6, check_every=64)
        tb = bt.tallies(0)
        with B.Simulation(nx, ny, nz, dx, V, dt_s=dt0, scheme=B.IT_UPWIND, dt_ladder=True, react_kappa=0.0625) as g:
            n = len(tr)
            g.schedule(np.tile(tr.x_cm, 4), np.tile(tr.y_cm, 4), np.tile(tr.let_keV_um, 4), np.tile(tr.b_cm, 4),
                       np.repeat(np.arange(4, dtype=np.int64) * P, n))
            g.run_to_completion(tol=1e-6, check_every=64)
            ts = g.tallies()
            log = g.dt_log()
            assert len(log) >= 2 and log[1][0] > 3 * P, log
            assert ts.steps == tb.steps and ts.dt_s == tb.dt_s
            for s in range(2):
                assert np.array_equal(bt.density(0, s), g.density(s))
            assert tb.f == pytest.approx(ts.f, abs=1e-7)
