"""FP64 reference of the surrogate MLP -- TEST INFRASTRUCTURE ONLY.

Only tests/ may import this module.  It restates, in plain numpy, the network
the CUDA library trains: 6 inputs, four hidden layers of 256 with SiLU
(x * sigmoid(x)), one output through a sigmoid so that f lies in (0, 1),
mean-squared error loss, and Adam (Kingma & Ba, ICLR 2015) on FP32 master
weights.  Parameters per member, in order:
    W1 [256][6], b1 [256], W2 [256][256], b2, W3 [256][256], b3,
    W4 [256][256], b4, W5 [1][256], b5 [1]
(W stored out-features x in-features).

``quant=True`` applies the precision points of the GPU path, while every sum
is FP64: weights rounded to bfloat16; every layer input (the normalised
inputs and each SiLU output, first rounded to float32) carried as the
two-term bfloat16 expansion hi + lo, hi = bf16(a), lo = bf16(a - hi), in the
forward pass and in the output layer's weight gradient; the one-term hi
part in the weight gradients of the hidden layers; the backward error
signals rounded to bfloat16 before they enter a matrix product.
``quant=False`` is plain FP64 (pinned against finite differences).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 256
N_IN = 6
SHAPES = [(HIDDEN, N_IN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,),
          (HIDDEN, HIDDEN), (HIDDEN,), (1, HIDDEN), (1,)]
N_PARAMS = int(sum(np.prod(s) for s in SHAPES))


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    The value is first rounded to float32 (the GPU rounds FP32 values), then
    the low 16 bits of the float32 pattern are rounded away."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    # NaN/Inf are passed through unchanged
    bad = ~np.isfinite(f)
    if np.any(bad):
        out = np.where(bad, f.astype(np.float64), out)
    return out


def bf16_split(x) -> np.ndarray:
    """The two-term bfloat16 expansion hi + lo of float32(x): hi = bf16(x),
    lo = bf16(x - hi) (the difference is exact in float32).  Represents
    float32(x) to within 2^-16 of |x| (one bf16 rounding of a residual at most
    2^-9 of |x|)."""
    f = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(f)
    return hi + bf16(f - hi)


def unpack(theta: np.ndarray):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, quant=False):
    """X: [B][6] normalised inputs.  Returns (fhat [B], cache): the cache
    holds the pre-activations, the layer inputs as the forward pass used them
    (hi + lo when quantised) and their one-term bf16 (hi) parts."""
    ident = lambda a: np.asarray(a, dtype=np.float64)
    q = bf16 if quant else ident
    qa = bf16_split if quant else ident
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5 = unpack(np.asarray(theta, dtype=np.float64))
    a = np.asarray(X, dtype=np.float64)
    A = qa(a)
    Zs, As, His = [], [A], [q(a)]
    for W, b in ((W1, b1), (W2, b2), (W3, b3), (W4, b4)):
        Z = A @ q(W).T + b
        s = silu(Z)
        A = qa(s)
        Zs.append(Z)
        As.append(A)
        His.append(q(s))
    z = A @ q(W5).T[:, 0] + b5[0]
    fhat = 1.0 / (1.0 + np.exp(-z))
    return fhat, (Zs, As, His, z)


def loss_and_grad(theta, X, y, quant=False):
    """Mean squared error (1/B) sum (fhat - y)^2 and its gradient."""
    q = bf16 if quant else (lambda a: np.asarray(a, dtype=np.float64))
    theta = np.asarray(theta, dtype=np.float64)
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5 = unpack(theta)
    fhat, (Zs, As, His, z) = forward(theta, X, quant)
    B = X.shape[0]
    loss = float(np.mean((fhat - y) ** 2))
    dz = 2.0 / B * (fhat - y) * fhat * (1.0 - fhat)          # through the output sigmoid
    gW5 = (dz @ As[4])[None, :]
    gb5 = np.array([dz.sum()])
    dA = np.outer(dz, q(W5)[0])
    grads = [None] * 8
    Ws = [W1, W2, W3, W4]
    for l in (3, 2, 1, 0):
        dZ = dA * dsilu(Zs[l])
        dZq = q(dZ)
        grads[2 * l] = dZq.T @ His[l]                            # dW [out][in], hi part of the input
        grads[2 * l + 1] = dZ.sum(axis=0)                        # db from the unrounded signal
        if l > 0:
            dA = dZq @ q(Ws[l])
    g = pack(grads + [gW5, gb5])
    return loss, g


class Adam:
    """Adam with bias correction on FP64 parameters (the master copy)."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
