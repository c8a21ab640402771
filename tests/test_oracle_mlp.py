"""Pins of the FP64 surrogate-network reference (no GPU needed): the
hand-written backward pass equals central finite differences, a linear
special case has its closed-form gradient, and Adam's first step moves each
parameter by lr against the sign of its gradient."""
import numpy as np

import oracle.mlp as mlp


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, width, depth, n_out, B = 5, 7, 3, 4, 6
    theta = rng.normal(0, 0.4, mlp.num_params(n_in, width, depth, n_out))
    x = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, (B, n_out))
    _, g = mlp.loss_and_grad(theta, x, t, n_in, width, depth, n_out)
    h = 1e-6
    for k in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        lp, _ = mlp.loss_and_grad(tp, x, t, n_in, width, depth, n_out)
        lm, _ = mlp.loss_and_grad(tm, x, t, n_in, width, depth, n_out)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-8 * max(1.0, abs(g[k]))


def test_linear_special_case_closed_form():
    # depth 0: y = x W + b, L = |y - t|^2 / (B n_out): dL/dW = 2 x^T (y - t) / (B n_out)
    rng = np.random.default_rng(1)
    n_in, n_out, B = 3, 2, 5
    theta = rng.normal(0, 1, n_in * n_out + n_out)
    x = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, (B, n_out))
    W, b = theta[:6].reshape(3, 2), theta[6:]
    y = x @ W + b
    _, g = mlp.loss_and_grad(theta, x, t, n_in, 0, 0, n_out)
    assert np.allclose(g[:6].reshape(3, 2), 2 * x.T @ (y - t) / (B * n_out), atol=1e-14)
    assert np.allclose(g[6:], 2 * (y - t).sum(0) / (B * n_out), atol=1e-14)


def test_adam_first_step_moves_by_lr():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)
