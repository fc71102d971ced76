"""Pins of the Adam oracle (Section 4.1; Kingma and Ba, Algorithm 1) by
closed forms of its update, independent of the oracle's own code."""

import numpy as np

from oracle.adam import adam_step


def test_first_step_moves_by_lr_times_the_sign():
    # bias correction makes m_hat = g and v_hat = g^2 at t = 1, so the step is
    # lr g / (|g| + eps)
    g = np.array([3.0, -0.02, 1e-3, -7.5])
    p, m, v = adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1, eps=1e-8)
    assert np.allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_constant_gradient_moves_lr_per_step():
    # with g constant, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2 exactly,
    # so every step moves lr g / (|g| + eps)
    g = np.array([0.5, -2.0])
    p, m, v = np.array([1.0, 1.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 11):
        p, m, v = adam_step(p, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
    assert np.allclose(p, 1.0 - 10 * 0.01 * np.sign(g), rtol=0, atol=1e-12)


def test_momentum_after_the_gradient_stops():
    # g1 = g, g2 = 0: m2 = 0.09 g, v2 = 0.000999 g^2,
    # step 2 = lr (0.09 / 0.19) / sqrt(0.000999 / 0.001999001) in units of sign(g)
    g = np.array([4.0])
    p, m, v = adam_step(np.zeros(1), g, np.zeros(1), np.zeros(1), 1, lr=1.0, eps=0.0)
    p2, _, _ = adam_step(p, np.zeros(1), m, v, 2, lr=1.0, eps=0.0)
    step2 = (0.09 / (1 - 0.81)) / np.sqrt(0.000999 / (1 - 0.999 ** 2))
    assert abs((p - p2)[0] - step2) <= 1e-12
    assert abs(step2 - 0.670064) <= 1e-5


def test_scale_invariance_and_box():
    rng = np.random.default_rng(3)
    g = rng.normal(size=50)
    a = adam_step(np.zeros(50), g, np.zeros(50), np.zeros(50), 1, lr=0.3, eps=0.0)[0]
    b = adam_step(np.zeros(50), 1000.0 * g, np.zeros(50), np.zeros(50), 1, lr=0.3, eps=0.0)[0]
    assert np.allclose(a, b, rtol=1e-14)
    c = adam_step(np.full(50, 0.5), g, np.zeros(50), np.zeros(50), 1, lr=0.3, lo=0.4, hi=0.6)[0]
    assert c.min() >= 0.4 and c.max() <= 0.6
    assert np.array_equal(c, np.clip(0.5 - 0.3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), 0.4, 0.6))


def test_per_parameter_learning_rates():
    g = np.array([1.0, 1.0, -1.0])
    lr = np.array([0.1, 0.2, 0.3])
    p = adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=lr, eps=0.0)[0]
    assert np.allclose(p, [-0.1, -0.2, 0.3])
