"""FP64 reference of the surrogate network: forward, mean-squared-error loss,
backward and one Adam update, written out layer by layer.

TEST INFRASTRUCTURE ONLY: used by tests/ and the benchmark's CPU baseline to
check the GPU kernels; nothing in the product path imports it.

The surrogate maps the rotated intrinsic coordinates x (4 numbers, the same
metric-eigenbasis point the RBF interpolant is evaluated at, Sec. II D) to
the interpolated columns F(x) (per-column standardised).  Network:

    h0 = x
    z_l = W_l h_{l-1} + b_l,  h_l = SiLU(z_l) = z_l * sigmoid(z_l)   (l = 1..L-1)
    y = W_L h_{L-1} + b_L

loss = mean over the batch and the outputs of (y - t)^2.  Gradients follow
the chain rule; SiLU'(z) = s(z) (1 + z (1 - s(z))) with s the logistic
function.  The optimiser is Adam (Kingma & Ba 2015, Algorithm 1) with bias
correction.

Parameters are kept as a list [(W_1, b_1), ..., (W_L, b_L)] with W_l of
shape [out, in]; `flatten` / `unflatten` give the flat order shared with
the GPU library: W_1 row-major, b_1, W_2, b_2, ...
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def shapes(n_in: int, hidden: int, n_hidden: int, n_out: int):
    """[(out, in)] of every layer."""
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def n_params(n_in: int, hidden: int, n_hidden: int, n_out: int) -> int:
    return sum(o * i + o for o, i in shapes(n_in, hidden, n_hidden, n_out))


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat, n_in: int, hidden: int, n_hidden: int, n_out: int):
    flat = np.asarray(flat, dtype=np.float64)
    out, p = [], 0
    for o, i in shapes(n_in, hidden, n_hidden, n_out):
        W = flat[p:p + o * i].reshape(o, i)
        p += o * i
        b = flat[p:p + o]
        p += o
        out.append((W.copy(), b.copy()))
    assert p == flat.size
    return out


def forward(params, x):
    """Returns (y, cache); cache = (inputs h_{l-1} and pre-activations z_l of
    every layer) for the backward pass."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if l < L - 1 else z
    return h, cache


def loss(y, t) -> float:
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(params, cache, y, t):
    """Gradients [(dW_l, db_l)] of the mean-squared-error loss."""
    B, K = y.shape
    g = 2.0 * (y - np.asarray(t, dtype=np.float64)) / (B * K)   # dloss/dy
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        h_in, z = cache[l]
        if l < len(params) - 1:
            g = g * silu_grad(z)             # through h_l = SiLU(z_l)
        grads[l] = (g.T @ h_in, g.sum(axis=0))
        g = g @ W                            # dloss/dh_{l-1}
    return grads


class Adam:
    """Adam with bias correction, one state pair per parameter array."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads, lr=None):
        lr = self.lr if lr is None else lr
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][j] + (1.0 - self.b1) * g
                v = self.b2 * self.v[l][j] + (1.0 - self.b2) * g * g
                self.m[l] = tuple(m if k == j else self.m[l][k] for k in range(2))
                self.v[l] = tuple(v if k == j else self.v[l][k] for k in range(2))
                new.append(p - lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            out.append((new[0], new[1]))
        return out
