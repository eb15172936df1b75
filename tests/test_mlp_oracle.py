"""Pins of the scorer network's CPU oracle (oracle/mlp.py): the backward pass
against central finite differences of the loss, the forward pass on a network
whose output is worked out by hand, and the bfloat16 rounding on known bit
patterns."""
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
