"""Pins of the scorer network's CPU oracle (oracle/mlp.py): the backward pass
against central finite differences of the loss, the forward pass on a network
whose output is worked out by hand, the bfloat16 rounding on known bit
patterns, and the forward pass with bfloat16 operands (the tensor-core
inference) on a hand-worked network and on values bfloat16 holds exactly."""
from __future__ import annotations

import numpy as np

from oracle import mlp as M


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    F, Hd, N = 5, 8, 7
    theta = rng.normal(0.0, 0.5, M.n_params(F, Hd))
    x = rng.normal(0.0, 1.0, (N, F))
    t = rng.normal(0.0, 1.0, N)
    g = M.grad(theta, x, t, Hd)
    h = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (M.loss(theta + e, x, t, Hd) - M.loss(theta - e, x, t, Hd)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_forward_of_a_hand_worked_network():
    # hidden width 2: h1 = relu([x0 - x1, x1 - x0]) = [|x0 - x1|, 0] for x0 > x1;
    # W2 = W3 = identity, biases 0, w4 = (1, 1), b4 = 0.5  ->  y = |x0 - x1| + 0.5
    F, Hd = 2, 2
    theta = np.concatenate([np.array([[1.0, -1.0], [-1.0, 1.0]]).ravel(), [0.0, 0.0],
                            np.eye(2).ravel(), [0.0, 0.0], np.eye(2).ravel(), [0.0, 0.0], [1.0, 1.0], [0.5]])
    x = np.array([[3.0, 1.0], [1.0, 4.0], [2.0, 2.0]])
    y, _ = M.forward(theta, x, Hd)
    assert np.allclose(y, [2.5, 3.5, 0.5], rtol=0, atol=0)


def test_bf16_rounding_on_known_values():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.140625, 1.0 + 2.0 ** -9], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, -2.5, 3.140625, 1.0], np.float32)
    assert np.array_equal(M.bf16_round(vals), want)


def test_bf16_operand_forward_rounds_each_layer_input():
    # x = (1, 2^-9) is exact in bfloat16; W1 sums both inputs into unit 0, so
    # h1 = (1 + 2^-9, 0).  Layer 2 takes h1 rounded (1 + 2^-9 -> 1), W2 = I;
    # layer 3 adds b3 = (2^-9, 0), W3 = I: h3 = (1 + 2^-9, 0), which the output
    # layer takes unrounded (w4 = (1, 1)).  Unrounded activations give 1 + 2^-8.
    F, Hd = 2, 2
    e = 2.0 ** -9
    theta = np.concatenate([np.array([[1.0, 0.0], [1.0, 0.0]]).ravel(), [0.0, 0.0],
                            np.eye(2).ravel(), [0.0, 0.0], np.eye(2).ravel(), [e, 0.0], [1.0, 1.0], [0.0]])
    x = np.array([[1.0, e]])
    assert M.forward_bf16_operands(theta, x, Hd)[0] == 1.0 + e
    assert M.forward(theta, x, Hd)[0][0] == 1.0 + 2 * e
    # an input that bfloat16 does not hold is rounded before the first layer
    x2 = np.array([[1.0 + e, 0.0]])
    assert M.forward_bf16_operands(theta, x2, Hd)[0] == 1.0 + e


def test_bf16_operand_forward_equals_forward_on_exact_values():
    # weights in {-1, 0, 1}, integer biases and inputs: every activation is an
    # integer below 256, which bfloat16 holds, so the rounding changes nothing
    rng = np.random.default_rng(5)
    F, Hd = 3, 4
    sz = M.sizes(F, Hd)
    parts = []
    for i, shp in enumerate(sz):
        if i in (1, 3, 5, 7):
            parts.append(rng.integers(-2, 3, shp).astype(np.float64).ravel())
        else:
            parts.append(rng.integers(-1, 2, shp).astype(np.float64).ravel())
    theta = np.concatenate(parts)
    x = rng.integers(-3, 4, (50, F)).astype(np.float64)
    y, acts = M.forward(theta, x, Hd)
    assert max(np.abs(a).max() for a in acts) < 256
    assert np.array_equal(M.forward_bf16_operands(theta, x, Hd), y)
