"""Tracks at an angle to the field (Fig. setup (a), Eq. angle) against the
oracle.  The deposit is FP64 arithmetic added once to the state, so FP32
states agree to one FP32 rounding (6e-8 of the value; 1e-6 of the maximum is
asserted) and FP64 states to 1e-12; the runs meet the bounds of the parallel
parity tests (densities 1e-4 of the maximum, f 1e-5)."""
import math

import numpy as np
import pytest

import oracle.oracle as o
from paper_1610_06749_gb300 import binding as B

pytestmark = pytest.mark.gpu

MU, DD, ALPHA = (1.73, 1.87), (0.037, 0.037), 1.6e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()


def _close(gpu, orc, tol, what=""):
    scale = np.max(np.abs(orc))
    err = np.max(np.abs(gpu.astype(np.float64) - orc)) / scale
    assert err <= tol, f"{what}: max abs error / max = {err:.3e} > {tol}"


TRACKS = dict(x=[0.0041, 0.0003], y=[0.0033, 0.0058], let=[50.0, 3.0], b=[1e-3, 6e-4])


@pytest.mark.parametrize("theta", [0.0, 0.4, 1.1, math.pi / 2])
@pytest.mark.parametrize("lat", [B.IT_PERIODIC, B.IT_ABSORBING])
@pytest.mark.parametrize("prec", [B.IT_FP32, B.IT_FP64])
def test_angled_deposit_matches_oracle(theta, lat, prec):
    nx, ny, nz, dx = 40, 30, 50, 2e-4
    th = [theta, 0.5 * theta]
    O = o.Oracle(nx, ny, nz, dx, 1e-9, lateral_bc=o.LATERAL_ABSORBING if lat == B.IT_ABSORBING else o.LATERAL_PERIODIC)
    r = O.deposit_angled(TRACKS["x"], TRACKS["y"], TRACKS["let"], TRACKS["b"], th)
    with B.Simulation(nx, ny, nz, dx, 200.0, dt_s=1e-9, lateral_bc=lat, precision=prec) as g:
        g.deposit_angled(TRACKS["x"], TRACKS["y"], TRACKS["let"], TRACKS["b"], th)
        tol = 1e-6 if prec == B.IT_FP32 else 1e-12
        for s in range(2):
            _close(g.density(s), O.density(s), tol, what=f"species {s}")
        np.testing.assert_allclose(g.tallies().released, [r, r], rtol=1e-12)


def test_angled_deposit_at_zero_is_the_parallel_deposit():
    nx, ny, nz, dx = 40, 30, 50, 2e-4
    with B.Simulation(nx, ny, nz, dx, 200.0, dt_s=1e-9) as a, B.Simulation(nx, ny, nz, dx, 200.0, dt_s=1e-9) as p:
        a.deposit_angled(TRACKS["x"], TRACKS["y"], TRACKS["let"], TRACKS["b"], [0.0, 0.0])
        p.deposit(TRACKS["x"], TRACKS["y"], TRACKS["let"], TRACKS["b"])
        for s in range(2):
            # the same FP64 sums in another order, rounded once to FP32
            _close(a.density(s), p.density(s).astype(np.float64), 2e-7)
        np.testing.assert_allclose(a.tallies().released, p.tallies().released, rtol=1e-13)


def test_tilted_track_run_matches_oracle():
    # a segment at 0.6 rad through a box with absorbing faces, 200 steps
    nx, ny, nz, dx, V = 48, 32, 40, 5e-4, 100.0
    npk = o.peak_track_density([100.0], [1e-3])
    dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=npk)
    O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V, lateral_bc=o.LATERAL_ABSORBING)
    O.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [100.0], [1e-3], [0.6])
    O.step(200)
    with B.Simulation(nx, ny, nz, dx, V, dt_s=dt, lateral_bc=B.IT_ABSORBING) as g:
        g.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [100.0], [1e-3], [0.6])
        g.step(200)
        for s in range(2):
            _close(g.density(s), O.density(s), 1e-4, what=f"species {s}")
        tg, to = g.tallies(), O.tallies()
        assert tg.f == pytest.approx(to.f, abs=1e-5)
        tot = to.released.sum()
        for name in ("collected_anode", "collected_cathode", "lost_lateral", "in_domain"):
            np.testing.assert_allclose(getattr(tg, name), getattr(to, name), rtol=0, atol=1e-5 * tot)


def test_track_parallel_to_the_electrodes_matches_oracle_and_jaffe_angle():
    # Eq. (angle) at pi/2: LET 1 keV/um, b = 10 um, E = 1000 V/cm, dx = b/5,
    # a track along x at mid-gap (periodic x), run to completion
    b, E, let, frac = 1e-3, 1000.0, 1.0, 5
    dx = b / frac
    nx, ny, nz = 4, 10 * frac, 40 * frac
    V = E * nz * dx
    dt = o.dt_rule(dx, V, nz * dx, MU, DD, ALPHA, n_peak=o.peak_track_density([let], [b]))
    O = o.Oracle(nx, ny, nz, dx, dt, mu=MU, D=DD, alpha=ALPHA, voltage_V=V)
    O.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [let], [b], [math.pi / 2])
    steps_o, done, _ = O.run_to_completion(1e-6, 100_000, 64)
    assert done
    with B.Simulation(nx, ny, nz, dx, V, dt_s=dt) as g:
        g.deposit_angled([0.5 * nx * dx], [0.5 * ny * dx], [let], [b], [math.pi / 2])
        steps_g = g.run_to_completion(tol=1e-6, max_steps=100_000, check_every=64)
        assert abs(steps_g - steps_o) <= 64   # the completion check may fall one interval apart
        fg, fo = g.tallies().f, O.tallies().f
        assert fg == pytest.approx(fo, abs=1e-5)
        fj = o.jaffe_angle(let, b, E, math.pi / 2, 0.5 * (MU[0] + MU[1]), 0.037, ALPHA)
        assert abs(fg - fj) < 3e-3


def test_angled_deposit_rejects_bad_angles():
    with B.Simulation(8, 8, 8, 5e-4, 100.0, dt_s=1e-9) as g:
        for bad in (-0.1, math.pi / 2 + 1e-9, float("nan")):
            with pytest.raises(B.ItError) as e:
                g.deposit_angled([1e-3], [1e-3], [1.0], [1e-3], [bad])
            assert e.value.code == B.IT_EINVAL
