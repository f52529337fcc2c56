"""FP64 oracle of the learned tuner's network -- TEST INFRASTRUCTURE ONLY.

The network is a 3-layer perceptron (input -> 64 -> 64 -> 1) with ReLU after the two hidden
layers and a linear output, trained on mean squared error -- the "small learned tuner" that maps
a configuration's features to predicted throughput.  (The paper's own tuner, Sect. 4.2.2, is a
measured search; the network is an added component and has no listing in the paper, so this
oracle follows the textbook definitions of the layers, the loss, back-propagation, SGD and Adam
(Kingma & Ba 2015, Algorithm 1).)

Flat parameter layout (shared with the CUDA kernels by convention only):
    [W1 (64 x D, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1)]
"""
from __future__ import annotations

import numpy as np

H = 64


def n_params(d: int) -> int:
    return H * d + H + H * H + H + H + 1


def unpack(p: np.ndarray, d: int):
    o = 0
    W1 = p[o:o + H * d].reshape(H, d); o += H * d
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H].reshape(1, H); o += H
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([W1.ravel(), b1.ravel(), W2.ravel(), b2.ravel(), W3.ravel(), b3.ravel()])


def forward(p, X, relu=True):
    """Return (prediction [N], cache).  X is [N, D]."""
    d = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, dtype=np.float64), d)
    act = (lambda z: np.maximum(z, 0.0)) if relu else (lambda z: z)
    z1 = X @ W1.T + b1
    h1 = act(z1)
    z2 = h1 @ W2.T + b2
    h2 = act(z2)
    y = (h2 @ W3.T + b3)[:, 0]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, t, relu=True) -> float:
    y, _ = forward(p, X, relu)
    return float(np.mean((y - t) ** 2))


def backward(p, X, t, relu=True):
    """Gradient of the mean squared error with respect to the flat parameters."""
    d = X.shape[1]
    n = X.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, dtype=np.float64), d)
    y, (X, z1, h1, z2, h2) = forward(p, X, relu)
    dy = (2.0 / n) * (y - t)                     # dL/dy
    gW3 = dy[None, :] @ h2                        # [1, 64]
    gb3 = np.array([dy.sum()])
    dh2 = dy[:, None] @ W3                        # [N, 64]
    dz2 = dh2 * (z2 > 0) if relu else dh2
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0) if relu else dh1
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def sgd_step(p, g, lr):
    return p - lr * g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
