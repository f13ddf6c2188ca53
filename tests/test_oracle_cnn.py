"""Pins for the oracle warm-start network.

- The convolution is checked against SciPy's 2-D correlation.
- Gradients are checked against central finite differences.
- Adam is checked against its closed-form first step.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def rand_theta(rng, scale=0.2):
    return rng.standard_normal(cnn.N_PARAMS) * scale


def test_parameter_count():
    assert cnn.N_PARAMS == 19105
    rng = np.random.default_rng(0)
    th = rand_theta(rng)
    assert np.array_equal(cnn.pack(cnn.unpack(th)), th)


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[bi, i], W[o, i], mode="same", boundary="fill", fillvalue=0) for i in range(3))
            assert np.allclose(y[bi, o], ref + b[o], atol=1e-12)


def test_identity_network_is_residual_identity():
    """With all weights zero the net outputs its input (the residual path alone)."""
    x = np.random.default_rng(2).standard_normal((3, 16, 32))
    y, _ = cnn.forward(np.zeros(cnn.N_PARAMS), x)
    assert np.array_equal(y, x)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    th = rand_theta(rng, 0.3)
    # Biases pushed positive so that few ReLUs sit at the kink.
    p = cnn.unpack(th)
    for k in ("b1", "b2", "b3"):
        p[k] = np.abs(p[k]) + 0.3
    th = cnn.pack(p)
    x = rng.standard_normal((2, 5, 6))
    t = rng.standard_normal((2, 5, 6))
    loss, g = cnn.loss_and_grad(th, x, t)
    idx = np.concatenate([rng.choice(cnn.N_PARAMS, 60, replace=False), [0, 320, 9567, 19104]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (cnn.loss_and_grad(th + e, x, t)[0] - cnn.loss_and_grad(th - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_closed_form():
    """At k = 1 the bias-corrected step is lr * g / (|g| + eps), i.e. almost lr * sign(g)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 2.0, 3.0, 4.0])
    new, m, v = cnn.adam_step(th, np.zeros(4), np.zeros(4), g, 1, lr=0.01, eps=1e-8)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
