"""Checkpoint and resume: a run stopped after k steps, its densities read out
(it_get_density) and set into a fresh context (it_set_density) with the
same time step, continues bitwise as the uninterrupted run; the resumed
context's tallies are the uninterrupted run's tallies of the remaining steps
(to FP64 summation order).  The transport step is the Appendix scheme of
Eq. theEquation; nothing in it depends on the step counter, so the state
(n+, n-) and dt are all a resume needs."""
import numpy as np
import pytest

from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1610_06749_gb300 import build
    build.build()


@pytest.mark.parametrize("scheme,bc,kernel", [
    (B.IT_LAX_WENDROFF, B.IT_PERIODIC, B.IT_KERNEL_AUTO),
    (B.IT_UPWIND, B.IT_ABSORBING, B.IT_KERNEL_AUTO),
    (B.IT_UPWIND, B.IT_PERIODIC, B.IT_KERNEL_SIMPLE),
])
def test_resumed_run_is_bitwise_the_uninterrupted_run(scheme, bc, kernel):
    nx, ny, nz, dx, V = 64, 48, 100, 5e-4, 200.0
    tr = synth.uniform_tracks(1610067495, 40, nx * dx, ny * dx, 10e-4)
    npk = B.it_peak_density(tr.let_keV_um, tr.b_cm)
    k, m = 60, 90
    kw = dict(n_peak_cm3=npk, scheme=scheme, lateral_bc=bc, kernel=kernel)
    with B.Simulation(nx, ny, nz, dx, V, **kw) as a:
        a.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        a.step(k)
        p_k, m_k = a.density(0), a.density(1)
        t_k = a.tallies()
        a.step(m)
        p_end, m_end = a.density(0), a.density(1)
        t_end = a.tallies()
        dt = t_end.dt_s
    with B.Simulation(nx, ny, nz, dx, V, **kw) as b:
        assert b.tallies().dt_s == dt
        b.set_density(p_k, m_k)
        b.step(m)
        assert np.array_equal(b.density(0), p_end)
        assert np.array_equal(b.density(1), m_end)
        t_b = b.tallies()
    assert t_b.steps == m
    scale = float(np.sum(t_end.released))
    for name in ("collected_anode", "collected_cathode", "lost_lateral"):
        want = getattr(t_end, name) - getattr(t_k, name)
        assert np.allclose(getattr(t_b, name), want, rtol=0, atol=1e-12 * scale), name
    assert abs(t_b.recombined - (t_end.recombined - t_k.recombined)) <= 1e-12 * scale
    # the resumed context's released charge is what was set: the in-domain
    # charge at the checkpoint
    assert np.allclose(t_b.released, t_k.in_domain, rtol=1e-12, atol=0)
