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


def round_bf16(a):
    """Round to the nearest bfloat16, ties to even, through FP32 (the values
    the kernels hold are FP32), returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _fp32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def forward_tc(w, X, rnd=round_bf16):
    """The forward pass in the operand precision of the tensor-core kernels:
    the inputs, the weight matrices and each hidden layer's ReLU output are
    rounded by `rnd` (bfloat16) before their product; biases are FP32;
    products and sums are wide. Returns Y and the cache of backward_tc."""
    layers = unpack(_fp32(w))
    a = rnd(X)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = a @ rnd(W) + b
        if i < 3:
            h = np.maximum(z, 0.0)
            cache.append((a, h))
            a = rnd(h)
        else:
            cache.append((a, None))
            a = z
    return a, cache


def loss_and_grad_tc(w, X, T, rnd=round_bf16):
    """loss_and_grad() in the operand precision of the training kernel
    (tensor-core products take BF16 operands and add wide): the forward of
    forward_tc; each weight gradient is the product of the layer's rounded
    input (the operand the forward used) with the rounded output gradient,
    and the bias gradient the sum of the rounded output gradient; the
    gradient passed down a layer is the product of the rounded output
    gradient with the rounded weights, masked by the ReLU. With rnd =
    identity this is loss_and_grad()."""
    Y, cache = forward_tc(w, X, rnd)
    T = np.asarray(T, dtype=np.float64)
    n = Y.shape[0]
    L = float(np.mean((Y - T) ** 2))
    d = 2.0 * (Y - T) / (n * Y.shape[1])
    layers = unpack(_fp32(w))
    grads = [None] * 4
    for i in range(3, -1, -1):
        dr = rnd(d)
        grads[i] = (cache[i][0].T @ dr, dr.sum(axis=0))
        if i > 0:
            d = (dr @ rnd(layers[i][0]).T) * (cache[i - 1][1] > 0)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return L, flat


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
