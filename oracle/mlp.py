"""CPU oracle of the learned candidate scorer -- TEST INFRASTRUCTURE ONLY.

Plain numpy FP64 forward and backward passes of the scorer network, written
from their definitions, so that the library's CUDA training kernels can be
checked against them.  Only ``tests/`` may import this module.

Network (three hidden layers of 128 units, ReLU):
    h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), h3 = relu(h2 W3 + b3),
    y  = h3 w4 + b4
Loss: mean squared error L = (1/N) sum_i (y_i - t_i)^2.
Parameters are packed in one vector in the order W1 (F x H, row-major),
b1 (H), W2 (H x H), b2, W3 (H x H), b3, w4 (H), b4 (1).
"""
from __future__ import annotations

import numpy as np

H = 128


def sizes(F: int, hidden: int = H) -> list[tuple[int, ...]]:
    return [(F, hidden), (hidden,), (hidden, hidden), (hidden,), (hidden, hidden), (hidden,), (hidden,), (1,)]


def unpack(theta: np.ndarray, F: int, hidden: int = H) -> list[np.ndarray]:
    out, o = [], 0
    for shp in sizes(F, hidden):
        k = int(np.prod(shp))
        out.append(theta[o:o + k].reshape(shp))
        o += k
    assert o == theta.size
    return out


def n_params(F: int, hidden: int = H) -> int:
    return sum(int(np.prod(s)) for s in sizes(F, hidden))


def forward(theta: np.ndarray, x: np.ndarray, hidden: int = H):
    """Prediction y [N] and the pre-activations needed by the backward pass."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, np.float64), x.shape[1], hidden)
    x = np.asarray(x, np.float64)
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3 + b3
    h3 = np.maximum(z3, 0.0)
    y = h3 @ w4 + b4[0]
    return y, (x, z1, h1, z2, h2, z3, h3)


def loss(theta: np.ndarray, x: np.ndarray, t: np.ndarray, hidden: int = H) -> float:
    y, _ = forward(theta, x, hidden)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(theta: np.ndarray, x: np.ndarray, t: np.ndarray, hidden: int = H) -> np.ndarray:
    """dL/dtheta by the chain rule, layer by layer from the output back."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, np.float64), x.shape[1], hidden)
    y, (x, z1, h1, z2, h2, z3, h3) = forward(theta, x, hidden)
    N = x.shape[0]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / N          # dL/dy
    g_w4 = h3.T @ dy
    g_b4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * (z3 > 0)                         # dL/dz3
    g_W3 = h2.T @ d3
    g_b3 = d3.sum(axis=0)
    d2 = (d3 @ W3.T) * (z2 > 0)
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (z1 > 0)
    g_W1 = x.T @ d1
    g_b1 = d1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (g_W1, g_b1, g_W2, g_b2, g_W3, g_b3, g_w4, g_b4)])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even) and back."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32)


def forward_bf16_operands(theta: np.ndarray, x: np.ndarray, hidden: int = H) -> np.ndarray:
    """Prediction when every product of a hidden layer takes bfloat16 operands:
    the weights W1, W2, W3, w4 and each hidden layer's input (the features, h1,
    h2) are rounded to bfloat16 (nearest, ties to even) before the product; the
    products, sums, biases and ReLU are exact (FP64).  The output layer takes
    h3 unrounded.  This is the arithmetic of a bfloat16 tensor-core product with
    a wide accumulator, written out."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, np.float64), x.shape[1], hidden)
    r = lambda a: bf16_round(np.asarray(a, np.float64)).astype(np.float64)
    h = np.asarray(x, np.float64)
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        h = np.maximum(r(h) @ r(W) + b, 0.0)
    return h @ r(w4) + b4[0]
