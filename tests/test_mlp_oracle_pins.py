"""Pins of the FP64 surrogate-MLP reference (oracle/mlp.py)."""
import math

import numpy as np
import pytest

import oracle.mlp as M
from paper_1610_06749_gb300 import synth


def _small_problem(seed=3, B=5):
    theta = synth.mlp_init(seed, 1)[0]
    u = synth.uniform01(seed + 11, B * 7).reshape(B, 7)
    X = 2.0 * u[:, :6] - 1.0
    y = u[:, 6]
    return theta, X, y


def test_parameter_count():
    assert M.N_PARAMS == 6 * 256 + 256 + 3 * (256 * 256 + 256) + 256 + 1 == 199425


def test_gradient_matches_central_differences_fp64():
    # analytic backward pass vs (L(theta + h e) - L(theta - h e)) / 2h on a
    # sample of parameters from every tensor
    theta, X, y = _small_problem()
    _, g = M.loss_and_grad(theta, X, y, quant=False)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in M.SHAPES])
    rng_pick = synth.uniform01(77, 40)
    for t in range(len(M.SHAPES)):
        for r in rng_pick[4 * (t % 10):4 * (t % 10) + 4]:
            i = int(offs[t] + r * (offs[t + 1] - offs[t]))
            h = 1e-6 * max(1.0, abs(theta[i]))
            tp, tm = theta.copy(), theta.copy()
            tp[i] += h
            tm[i] -= h
            fd = (M.loss_and_grad(tp, X, y)[0] - M.loss_and_grad(tm, X, y)[0]) / (2 * h)
            # finite differences carry ~eps*L/h ~ 1e-11 of rounding noise
            assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 5e-11, (t, i, g[i], fd)


def test_silu_derivative_matches_central_differences():
    z = np.linspace(-8, 8, 41)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.dsilu(z), fd, rtol=1e-7, atol=1e-10)


def test_bf16_rounding_matches_torch():
    # an independent implementation: torch's float32 -> bfloat16 conversion
    torch = pytest.importorskip("torch")
    u = synth.uniform01(5, 2000)
    x = np.concatenate([(u - 0.5) * 10.0 ** np.linspace(-6, 6, 2000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


def test_bf16_split_two_term_expansion():
    # hi + lo with hi = bf16(x), lo = bf16(x - hi): torch computes the same two
    # roundings independently; the pair carries float32(x) to within 2^-16 of
    # |x| and exactly when x needs at most 16 significant bits
    torch = pytest.importorskip("torch")
    u = synth.uniform01(9, 3000)
    x = (u - 0.5) * 10.0 ** np.linspace(-5, 5, 3000)
    f = torch.tensor(x, dtype=torch.float32)
    hi = f.to(torch.bfloat16)
    lo = (f - hi.to(torch.float32)).to(torch.bfloat16)
    ref = hi.to(torch.float64).numpy() + lo.to(torch.float64).numpy()
    got = M.bf16_split(x)
    np.testing.assert_array_equal(got, ref)
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(got - x32) <= 2.0 ** -16 * np.abs(x32))
    exact = np.array([1.0 + 2 ** -15, -3.0 * (1 + 2 ** -13), 0.0, 2 ** -20 * (1 + 2 ** -10)])
    np.testing.assert_array_equal(M.bf16_split(exact), exact)


def test_adam_first_step_moves_by_lr_times_sign():
    # after the first step m_hat / sqrt(v_hat) = g/|g|: the update is lr*sign(g)
    a = M.Adam(3, lr=0.01)
    p = a.step(np.array([1.0, 2.0, 3.0]), np.array([0.5, -4.0, 1e-3]))
    g = np.array([0.5, -4.0, 1e-3])
    want = np.array([1.0, 2.0, 3.0]) - 0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(p, want, rtol=1e-14)


def test_quantised_forward_is_close_to_fp64_and_learns_nothing_wrong():
    theta, X, y = _small_problem(B=64)
    f0, _ = M.forward(theta, X, quant=False)
    f1, _ = M.forward(theta, X, quant=True)
    assert np.all((f0 > 0) & (f0 < 1))
    assert np.max(np.abs(f0 - f1)) < 2e-2          # bfloat16 weights, two-term bfloat16 activations
    # a few Adam steps on the quantised gradient lower the loss
    opt = M.Adam(theta.size, lr=1e-3)
    l0 = M.loss_and_grad(theta, X, y, quant=True)[0]
    for _ in range(60):
        _, g = M.loss_and_grad(theta, X, y, quant=True)
        theta = opt.step(theta, g)
    assert M.loss_and_grad(theta, X, y, quant=True)[0] < 0.6 * l0
