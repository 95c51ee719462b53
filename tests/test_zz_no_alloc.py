"""it_step_noalloc -- the step for callers that may not allocate device memory.

Such callers (code that only receives buffers from another framework's memory
pool, services that must not allocate after start-up) call it_step_noalloc
with their own input/output buffers; the kernel's tally partials live in a
fixed static device array instead of memory the library would allocate.
This checks, through the C ABI, that two calls in a row reproduce what the
context path (it_create + it_step + it_tallies) computes for the same two
steps.  The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu

IDX = ["recombined", "anode+", "anode-", "cathode+", "cathode-", "lateral+", "lateral-"]


def _vec(t):
    return np.array([t.recombined, t.collected_anode[0], t.collected_anode[1], t.collected_cathode[0],
                     t.collected_cathode[1], t.lost_lateral[0], t.lost_lateral[1]])


@pytest.mark.parametrize("bc", [B.IT_PERIODIC, B.IT_ABSORBING])
def test_step_noalloc_matches_context_step_on_two_calls(bc):
    import torch
    from paper_1610_06749_gb300 import build
    build.build()
    nx, ny, nz, dx, V = 64, 48, 40, 5e-4, 200.0
    tr = synth.uniform_tracks(77, 20, nx * dx, ny * dx, 1e-3)
    npk = B.it_peak_density(tr.let_keV_um, tr.b_cm)
    p = B.it_params_default(gap_cm=nz * dx, voltage_V=V, n_peak_cm3=npk, lateral_bc=bc,
                            kernel=B.IT_KERNEL_SIMPLE)
    dt = B.it_auto_dt(p, dx)

    # reference: the context path
    with B.Simulation(nx, ny, nz, dx, V, dt_s=dt, lateral_bc=bc, kernel=B.IT_KERNEL_SIMPLE) as sim:
        sim.deposit(tr.x_cm, tr.y_cm, tr.let_keV_um, tr.b_cm)
        n0 = (sim.density(0), sim.density(1))
        t0 = sim.tallies()
        sim.step(1)
        t1 = sim.tallies()
        d1 = (sim.density(0), sim.density(1))
        sim.step(1)
        t2 = sim.tallies()
        d2 = (sim.density(0), sim.density(1))
    released = t0.released.sum()

    dev = torch.device("cuda", 0)
    a = [torch.from_numpy(n0[0]).to(dev), torch.from_numpy(n0[1]).to(dev)]
    b = [torch.empty_like(a[0]), torch.empty_like(a[1])]
    tal = torch.full((7,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    expect = [(d1, _vec(t1) - _vec(t0)), (d2, _vec(t2) - _vec(t1))]
    for call in range(2):
        B.it_step_noalloc(nx, ny, nz, dx, dt, p, a[0].data_ptr(), a[1].data_ptr(), b[0].data_ptr(),
                          b[1].data_ptr(), tal.data_ptr(), stream)
        torch.cuda.synchronize()
        want_d, want_t = expect[call]
        for s in range(2):
            got = b[s].cpu().numpy()
            # same kernel code on the same inputs: the densities agree bitwise
            assert np.array_equal(got, want_d[s]), f"call {call} species {s}"
        got_t = tal.cpu().numpy()
        assert np.all(np.isfinite(got_t))
        np.testing.assert_allclose(got_t, want_t, rtol=0, atol=1e-9 * released,
                                   err_msg=f"call {call}: tallies {IDX}")
        a, b = b, a          # this call's output is the next call's input
