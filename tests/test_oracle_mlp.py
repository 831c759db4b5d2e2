"""Pins of the oracle's correction network: finite-difference gradients, the
ReLU kink, Adam against its closed-form first step, and bf16 rounding against
exactly representable values."""
import numpy as np
import pytest

from oracle import mlp as M


def _net(rng, nin=7, H=5):
    return (rng.standard_normal((H, nin)), rng.standard_normal(H) * 0.1,
            rng.standard_normal((nin, H)), rng.standard_normal(nin) * 0.1)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    W1, b1, W2, b2 = _net(rng)
    X = rng.standard_normal((9, 7))
    T = rng.standard_normal((9, 7))
    loss, grads = M.loss_and_grads(W1, b1, W2, b2, X, T)
    params = [W1, b1, W2, b2]
    h = 1e-6
    for p, g in zip(params, grads):
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[idx]
            p[idx] = old + h
            lp, _ = M.loss_and_grads(*params, X, T)
            p[idx] = old - h
            lm, _ = M.loss_and_grads(*params, X, T)
            p[idx] = old
            assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-6 * max(1.0, abs(g[idx]))


def test_loss_is_mean_squared_error_and_relu_kills_negative_units():
    W1 = np.array([[1.0, 0.0], [-1.0, 0.0]])
    b1 = np.zeros(2)
    W2 = np.eye(2)
    b2 = np.zeros(2)
    X = np.array([[2.0, 5.0]])
    a1, h1, y = M.forward(W1, b1, W2, b2, X)
    assert np.allclose(h1, [[2.0, 0.0]]) and np.allclose(y, [[2.0, 0.0]])
    loss, (dW1, db1, dW2, db2) = M.loss_and_grads(W1, b1, W2, b2, X, np.zeros((1, 2)))
    assert loss == pytest.approx(4.0)
    assert np.allclose(dW1[1], 0.0) and db1[1] == 0.0      # dead unit gets no gradient


def test_adam_first_step_is_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    M.adam_step(p, g, m, v, t=1, lr=0.01, eps=0.0)
    # first step: mhat = g, vhat = g^2  ->  update = lr * sign(g)
    assert np.allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01])


def test_bf16_rounding():
    vals = np.array([1.0, -0.5, 3.0, 1.0 + 2 ** -7], dtype=np.float32)
    assert np.array_equal(M.bf16_round(vals), vals.astype(np.float64))
    # 1 + 2^-9 is below half an ulp of bf16 at 1 (2^-8): rounds to 1; 1 + 3*2^-9 rounds up to 1 + 2^-7
    assert M.bf16_round(np.float32(1 + 2 ** -9)) == 1.0
    assert M.bf16_round(np.float32(1 + 3 * 2 ** -9)) == 1.0 + 2 ** -7


def test_adam_constant_gradient_keeps_bias_corrected_moments_exact():
    # with a constant gradient g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the
    # bias-corrected moments are g and g^2 at every step and each update is lr * sign(g)
    # (eps = 0); b1 != b2, non-default, so a swapped or mis-indexed correction shows
    g = np.array([0.5, -4.0, 1e-3, 7.0])
    p = [np.array([1.0, -2.0, 3.0, 0.0])]
    m, v = [np.zeros(4)], [np.zeros(4)]
    for t in range(1, 6):
        M.adam_step(p, [g.copy()], m, v, t=t, lr=0.01, beta1=0.8, beta2=0.95, eps=0.0)
        assert np.allclose(p[0], np.array([1.0, -2.0, 3.0, 0.0]) - 0.01 * t * np.sign(g), atol=1e-15)
        assert np.allclose(m[0], (1 - 0.8 ** t) * g, rtol=1e-14)
        assert np.allclose(v[0], (1 - 0.95 ** t) * g * g, rtol=1e-14)


def test_adam_second_step_after_a_sign_flip_follows_the_closed_form():
    # g then -g: m_2 = -(1 - b1)^2 g, so mhat_2 = -(1 - b1) g / (1 + b1); v_2 = (1 - b2^2) g^2,
    # so vhat_2 = g^2; the second update is +lr (1 - b1) / (1 + b1) sign(g)
    b1, b2, lr = 0.7, 0.9, 0.05
    g = np.array([2.0, -0.25, 3.0])
    p0 = np.array([0.5, 0.5, -1.0])
    p = [p0.copy()]
    m, v = [np.zeros(3)], [np.zeros(3)]
    M.adam_step(p, [g.copy()], m, v, t=1, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    M.adam_step(p, [-g], m, v, t=2, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    expect = p0 - lr * np.sign(g) + lr * (1 - b1) / (1 + b1) * np.sign(g)
    assert np.allclose(p[0], expect, atol=1e-15)
