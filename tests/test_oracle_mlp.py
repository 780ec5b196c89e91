"""Pins of the CPU surrogate-MLP oracle: GELU against its closed forms and
the normal distribution, the backward pass against central finite
differences, a one-layer case against least squares algebra, and Adam
against a hand-worked first step."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import mlp as M


def test_gelu_closed_forms():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # x * Phi(x): Phi(1) = 0.841344746068543 (standard normal table)
    assert abs(M.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-12
    assert abs(M.gelu(np.array([-1.0]))[0] + 1.0 * (1 - 0.841344746068543)) < 1e-12
    x = np.linspace(-6, 6, 25)
    assert np.allclose(M.gelu(x) - M.gelu(-x), x)  # x Phi(x) + x Phi(-x) = x
    assert abs(M.gelu(np.array([12.0]))[0] - 12.0) < 1e-12


def test_gelu_grad_is_derivative():
    x = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(x), fd, atol=1e-8)
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def test_backward_matches_finite_differences():
    dims = (8, 6, 5, 4, 1)
    p = M.init_params(3, dims=dims, n_in=8)
    for k in p:
        if k.startswith("b"):
            p[k] = np.random.default_rng(len(k)).standard_normal(p[k].shape) * 0.1
    rng = np.random.default_rng(4)
    X = rng.standard_normal((11, 8))
    t = rng.standard_normal(11)
    g = M.backward(p, X, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, X, t)
            flat[idx] = old - h
            lm = M.loss(p, X, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) < 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_single_linear_layer_gradient_is_least_squares():
    """With one layer (no GELU) the gradient is the least-squares normal
    equation residual 2/n X^T (X w + b - t)."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((20, 5))
    t = rng.standard_normal(20)
    p = {"W1": rng.standard_normal((1, 5)), "b1": np.array([0.3])}
    g = M.backward(p, X, t)
    r = X @ p["W1"][0] + 0.3 - t
    assert np.allclose(g["W1"][0], 2.0 / 20 * X.T @ r)
    assert np.allclose(g["b1"][0], 2.0 / 20 * r.sum())


def test_adam_first_step_moves_by_lr_times_sign():
    """After one step from zero moments, m_hat = g and v_hat = g^2, so each
    parameter moves by lr * g / (|g| + eps) (Kingma and Ba, Sec. 2)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    M.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-9)


def test_bf16_round():
    assert M.bf16_round(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert M.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert M.bf16_round(np.array([-3.0]))[0] == -3.0
