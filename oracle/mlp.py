"""Warm-start network of the learned GMRES start — oracle (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline use this
module; the library never does.

The network maps per-DOF features to the density at that DOF (the learned
initial guess of GMRES, Algorithm 1 Step 4, from a zero start otherwise):

    z1 = W1 x + b1,   a1 = tanh(z1)            (width 256)
    z2 = W2 a1 + b2,  a2 = tanh(z2)            (width 256)
    y  = W3 a2 + b3 + WL x                      (one output)

WL is a linear skip from the inputs to the output.  W1, W2, W3 take part in
every product rounded to bfloat16 (round to nearest, ties to even, of the FP32
master value); WL, the activations, biases and all sums are kept in higher
precision (FP32 on the GPU, FP64 here), so that the linear part of the map is
resolved beyond bfloat16 precision.  Gradients are those of
the loss with respect to the rounded weights, applied to the FP32 masters.

Loss: L = 1/(2n) sum_i (y_i - t_i)^2.
Optimiser: Adam (Kingma & Ba, "Adam: A method for stochastic optimization",
ICLR 2015, Algorithm 1) with bias-corrected moments.
"""
from __future__ import annotations

import numpy as np


def bf16_round(w: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float64.  bfloat16 keeps the top 16 bits of the float32 pattern."""
    f = np.ascontiguousarray(w, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


class Params:
    """FP32 master parameters (held here as float64 copies of float32 values)."""

    def __init__(self, W1, b1, W2, b2, W3, b3, WL=None):
        self.W1, self.b1 = np.asarray(W1, np.float64), np.asarray(b1, np.float64)
        self.W2, self.b2 = np.asarray(W2, np.float64), np.asarray(b2, np.float64)
        self.W3, self.b3 = np.asarray(W3, np.float64), np.asarray(b3, np.float64)
        n_in = self.W1.shape[1]
        self.WL = np.zeros((1, n_in)) if WL is None else np.asarray(WL, np.float64).reshape(1, n_in)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2,
                               self.W3.ravel(), self.b3, self.WL.ravel()])

    @classmethod
    def from_flat(cls, v, n_in, width):
        v = np.asarray(v, np.float64)
        sizes = [width * n_in, width, width * width, width, width, 1, n_in]
        parts = np.split(v, np.cumsum(sizes)[:-1])
        return cls(parts[0].reshape(width, n_in), parts[1], parts[2].reshape(width, width),
                   parts[3], parts[4].reshape(1, width), parts[5], parts[6].reshape(1, n_in))


def forward(P: Params, X: np.ndarray, bf16: bool = True):
    """Network output for the rows of X (n x n_in) and the activations."""
    rw = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = rw(P.W1), rw(P.W2), rw(P.W3)
    z1 = X @ W1.T + P.b1
    a1 = np.tanh(z1)
    z2 = a1 @ W2.T + P.b2
    a2 = np.tanh(z2)
    y = (a2 @ W3.T)[:, 0] + P.b3[0] + (X @ P.WL.T)[:, 0]
    return y, (X, a1, a2, W1, W2, W3)


def loss_and_grad(P: Params, X: np.ndarray, t: np.ndarray, bf16: bool = True):
    """L = 1/(2n) sum (y - t)^2 and dL/d(parameters) by the chain rule."""
    n = X.shape[0]
    y, (X, a1, a2, W1, W2, W3) = forward(P, X, bf16)
    e = y - t
    L = 0.5 * float(e @ e) / n
    dy = e / n                                  # dL/dy_i
    gW3 = dy[None, :] @ a2                      # (1 x width)
    gb3 = np.array([dy.sum()])
    da2 = dy[:, None] * W3                      # (n x width)
    dz2 = da2 * (1.0 - a2 * a2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    da1 = dz2 @ W2
    dz1 = da1 * (1.0 - a1 * a1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    gWL = dy[None, :] @ X
    return L, Params(gW1, gb1, gW2, gb2, gW3, gb3, gWL)


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
