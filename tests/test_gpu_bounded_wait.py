"""The step kernel's bounded waits, made to run out on purpose without a
fault.

The z-march kernel's plane ring waits on an mbarrier per slot.  With the
test hook it_test_withhold_load the first ring load of every CTA is never
issued, so nothing ever completes that barrier phase: each warp's first wait
runs out after the it_set_wait_limit limit, the CTA drains the loads it did
issue (with the full bound) and returns, and the context's device error flag
makes the next it_tallies fail with IT_ETIMEOUT.  it_reset clears the flag
and the same context then steps exactly like a fresh one.  No load is left
in flight and no memory outside the state is touched.
"""
import time

import numpy as np
import pytest

from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()


def _setup():
    nx, ny, nz, dx, V = 64, 48, 40, 5e-4, 200.0
    tr = synth.uniform_tracks(31, 12, nx * dx, ny * dx, 1e-3)
    npk = B.it_peak_density(tr.let_keV_um, tr.b_cm)
    return (nx, ny, nz, dx, V, npk), tr


def test_a_short_wait_limit_runs_out_and_the_context_recovers():
    (nx, ny, nz, dx, V, npk), tr = _setup()
    with B.Simulation(nx, ny, nz, dx, V, n_peak_cm3=npk, kernel=B.IT_KERNEL_ZMARCH) as g, \
            B.Simulation(nx, ny, nz, dx, V, n_peak_cm3=npk, kernel=B.IT_KERNEL_ZMARCH) as ref:
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        B.it_set_wait_limit(g.h, 1 << 20)          # about 0.5 ms at 2 GHz
        B.it_test_withhold_load(g.h, True)
        t0 = time.perf_counter()
        g.step(3)
        with pytest.raises(B.ItError) as e:
            g.tallies()
        assert e.value.code == B.IT_ETIMEOUT
        # three launches that each gave up after ~2^20 cycles, not 2^32
        assert time.perf_counter() - t0 < 5.0
        # the flag stays raised until the context is reset
        with pytest.raises(B.ItError):
            g.tallies()
        B.it_test_withhold_load(g.h, False)
        g.reset()
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.step(40)
        ref.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        ref.step(40)
        tg, tr_ = g.tallies(), ref.tallies()
        for s in range(2):
            assert np.array_equal(g.density(s), ref.density(s))
        assert tg.f == tr_.f and tg.recombined == tr_.recombined and tg.steps == 40


def test_a_limit_well_above_the_load_time_never_runs_out():
    (nx, ny, nz, dx, V, npk), tr = _setup()
    with B.Simulation(nx, ny, nz, dx, V, n_peak_cm3=npk, kernel=B.IT_KERNEL_ZMARCH) as g:
        B.it_set_wait_limit(g.h, 1 << 24)          # about 8 ms, far above a plane's load time
        g.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        g.step(200)
        t = g.tallies()
        assert t.steps == 200 and np.isfinite(t.f)
        B.it_set_wait_limit(g.h, 0)                # back to the default


def test_wait_limit_and_hook_arguments():
    (nx, ny, nz, dx, V, npk), _ = _setup()
    with B.Simulation(nx, ny, nz, dx, V, n_peak_cm3=npk, kernel=B.IT_KERNEL_SIMPLE) as g:
        with pytest.raises(B.ItError) as e:
            B.it_set_wait_limit(g.h, -1)
        assert e.value.code == B.IT_EINVAL
        with pytest.raises(B.ItError) as e:
            B.it_test_withhold_load(g.h, True)
        assert e.value.code == B.IT_ESTATE
