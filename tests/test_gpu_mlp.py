"""The surrogate network's CUDA forward, backward and Adam kernels against the
FP64 reference (oracle/mlp.py at the same bfloat16 quantisation points)."""
import numpy as np
import pytest

import oracle.mlp as M
from paper_1610_06749_gb300 import binding as B
from paper_1610_06749_gb300 import synth

pytestmark = pytest.mark.gpu
MEMBERS = 3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1610_06749_gb300 import build
    build.build()
    B.lib()


def _net(seed=11, members=MEMBERS, max_batch=512):
    h = B.it_mlp_create(members, max_batch)
    theta = synth.mlp_init(seed, members)
    for m in range(members):
        B.it_mlp_set_params(h, m, theta[m])
    B.it_mlp_set_normalization(h, np.zeros(6), np.ones(6))
    # the oracle gets the same FP32 master values
    return h, theta.astype(np.float32).astype(np.float64)


def _data(seed, n):
    u = synth.uniform01(seed, n * 7).reshape(n, 7)
    X = 2.0 * u[:, :6] - 1.0
    y = 0.05 + 0.9 * u[:, 6]
    return X.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)


def test_forward_matches_reference():
    h, theta = _net()
    try:
        X, _ = _data(21, 300)
        mean, spread, per = B.it_mlp_predict(h, MEMBERS, X)
        for m in range(MEMBERS):
            ref, _ = M.forward(theta[m], X, quant=True)
            # measured: <= 3e-6; the members' FP32 tensor-core sums and the
            # reference's FP64 sums round the same bf16 points differently
            # only where a value sits on a rounding boundary
            print(f"forward member {m}: max abs {np.max(np.abs(per[:, m] - ref)):.3e}")
            assert np.max(np.abs(per[:, m] - ref)) < 1e-4
        assert np.allclose(mean, per.mean(axis=1)) and np.allclose(spread, per.max(axis=1) - per.min(axis=1))
    finally:
        B.it_mlp_destroy(h)


def test_gradients_match_reference():
    h, theta = _net()
    try:
        X, y = _data(22, 200)
        loss, g = B.it_mlp_loss_grad(h, MEMBERS, X, y)
        offs = np.cumsum([0] + [int(np.prod(s)) for s in M.SHAPES])
        for m in range(MEMBERS):
            lref, gref = M.loss_and_grad(theta[m], X, y, quant=True)
            print(f"loss member {m}: {loss[m]:.9e} vs {lref:.9e}")
            assert loss[m] == pytest.approx(lref, rel=1e-4)
            for t in range(len(M.SHAPES)):
                a, b = g[m, offs[t]:offs[t + 1]].astype(np.float64), gref[offs[t]:offs[t + 1]]
                err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
                print(f"grad member {m} tensor {t}: normwise {err:.3e}")
                # measured: <= 2.6e-4 per tensor
                assert err < 1e-3, (m, t, err)
    finally:
        B.it_mlp_destroy(h)


def test_adam_step_matches_reference():
    h, theta = _net(members=1)
    try:
        X, y = _data(23, 128)
        lr = 1e-3
        _, g = B.it_mlp_loss_grad(h, 1, X, y)
        B.it_mlp_adam_step(h, lr)
        p_gpu = B.it_mlp_get_params(h, 0).astype(np.float64)
        # Adam on the GPU's own gradient, in FP64: the update rule itself
        opt = M.Adam(theta[0].size, lr=lr)
        p_ref = opt.step(theta[0], g[0].astype(np.float64))
        assert np.max(np.abs(p_gpu - p_ref)) < 1e-6
        # and the direction agrees with the FP64 reference gradient where it is not tiny
        _, gref = M.loss_and_grad(theta[0], X, y, quant=True)
        big = np.abs(gref) > 1e-2 * np.abs(gref).max()
        assert np.mean(np.sign(p_gpu[big] - theta[0][big]) == -np.sign(gref[big])) > 0.99
    finally:
        B.it_mlp_destroy(h)


def test_training_learns_a_smooth_target_and_is_reproducible():
    X, _ = _data(24, 4096)
    w = np.array([0.8, -0.5, 0.3, 0.2, -0.4, 0.6])
    y = 1.0 / (1.0 + np.exp(-(X @ w)))
    params = []
    for _ in range(2):
        h, _ = _net(seed=5)
        try:
            B.it_mlp_set_data(h, X, y)
            loss = B.it_mlp_train(h, 40, 256, 1e-3, seed=99)
            assert loss[-1] < 0.05 * loss[0]
            params.append(B.it_mlp_get_params(h, 1))
        finally:
            B.it_mlp_destroy(h)
    assert np.array_equal(params[0], params[1])
