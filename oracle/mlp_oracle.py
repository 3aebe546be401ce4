"""Oracle of the learned near-surface gradient closure (test infrastructure).

TEST INFRASTRUCTURE ONLY: plain FP64 numpy statement of the multilayer
perceptron that the CUDA library trains and evaluates on tensor cores. The
paper has no closure; it motivates one: IBM underestimates the velocity
gradients, hence the dissipation, inside its diffused interface (Sec. 3.2,
Sec. 4). Network: 85 inputs -> 64 -> 64 -> 64 (ReLU) -> 9 outputs, MSE loss
averaged over samples and outputs, Adam.

Flat parameter layout (shared convention with the library's C ABI, each
W_l stored [in][out] row-major, then its bias):
    W1 (85x64), b1 (64), W2 (64x64), b2, W3 (64x64), b3, W4 (64x9), b4 (9).
"""
from __future__ import annotations

import numpy as np

SIZES = [85, 64, 64, 64, 9]


def n_params() -> int:
    return sum(SIZES[i] * SIZES[i + 1] + SIZES[i + 1] for i in range(4))


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = [], 0
    for i in range(4):
        a, b = SIZES[i], SIZES[i + 1]
        W = w[o:o + a * b].reshape(a, b)
        o += a * b
        bias = w[o:o + b]
        o += b
        out.append((W, bias))
    return out


def init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (seeded numpy; an input, not method)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(4):
        a, b = SIZES[i], SIZES[i + 1]
        parts.append(rng.standard_normal(a * b) * np.sqrt(2.0 / a))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def forward(w, X):
    """Returns outputs Y (n,9) and the cache (inputs of every layer and the
    pre-activations) for the backward pass."""
    layers = unpack(w)
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ W + b
        cache.append((h, z))
        h = np.maximum(z, 0.0) if i < 3 else z
    return h, cache


def loss_and_grad(w, X, T):
    """MSE loss L = mean((Y - T)^2) over samples and outputs and dL/dw by
    the chain rule."""
    Y, cache = forward(w, X)
    T = np.asarray(T, dtype=np.float64)
    n = Y.shape[0]
    L = float(np.mean((Y - T) ** 2))
    d = 2.0 * (Y - T) / (n * Y.shape[1])
    layers = unpack(w)
    grads = [None] * 4
    for i in range(3, -1, -1):
        h, z = cache[i]
        if i < 3:
            d = d * (z > 0)
        W, _ = layers[i]
        grads[i] = (h.T @ d, d.sum(axis=0))
        d = d @ W.T
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return L, flat


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015), t counted from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def train(w, X, T, epochs, batch, lr):
    """Sequential mini-batches over the given (pre-shuffled) samples."""
    w = np.array(w, dtype=np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    t = 0
    n = X.shape[0]
    for _ in range(epochs):
        for s in range(0, n, batch):
            t += 1
            _, g = loss_and_grad(w, X[s:s + batch], T[s:s + batch])
            w, m, v = adam(w, g, m, v, t, lr)
    return w
