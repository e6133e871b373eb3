"""Pins of the network oracle (finite differences, closed forms, bf16 rounding)."""
import math

import numpy as np
import pytest
from scipy.special import erf


@pytest.fixture(scope="module")
def M():
    from oracle import mlp

    return mlp


def test_gelu_and_its_derivative(M):
    z = np.linspace(-6, 6, 241)
    # Phi(z) = (1 + erf(z/sqrt2))/2 is the standard normal CDF
    from scipy.stats import norm

    assert np.abs(M.gelu(z) - z * norm.cdf(z)).max() < 1e-15
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.abs(M.gelu_grad(z) - fd).max() < 1e-8


def test_bf16_rounding(M):
    # exactly representable values pass, halfway cases round to even
    assert M.bf16_round(np.array([1.0, -2.5, 0.0]))[1] == -2.5
    one = 1.0
    ulp = 2.0 ** -7
    assert M.bf16_round(np.array([one + ulp / 2]))[0] == one          # tie -> even (1.0)
    assert M.bf16_round(np.array([one + 1.5 * ulp]))[0] == one + 2 * ulp  # tie -> even
    assert M.bf16_round(np.array([one + 0.6 * ulp]))[0] == one + ulp
    rng = np.random.default_rng(0)
    x = rng.standard_normal(1000)
    r = M.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * 1.0001)


def test_gradients_by_finite_differences(M):
    rng = np.random.default_rng(1)
    shapes = M.layer_shapes(4, 8, 2, 6)
    n = sum(o * i + o for o, i in shapes)
    p = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((5, 4))
    T = rng.standard_normal((5, 6))
    mask = (rng.uniform(size=(5, 6)) > 0.3).astype(float)
    loss, g = M.loss_and_grads(p, X, T, mask, shapes)
    for k in rng.choice(n, 25, replace=False):
        e = np.zeros(n)
        e[k] = 1e-6
        lp, _ = M.loss_and_grads(p + e, X, T, mask, shapes)
        lm, _ = M.loss_and_grads(p - e, X, T, mask, shapes)
        assert abs((lp - lm) / 2e-6 - g[k]) < 1e-7 * max(1.0, abs(g[k]))


def test_masked_entries_do_not_contribute(M):
    rng = np.random.default_rng(2)
    shapes = M.layer_shapes(4, 8, 2, 6)
    n = sum(o * i + o for o, i in shapes)
    p = rng.standard_normal(n) * 0.3
    X = rng.standard_normal((3, 4))
    T = rng.standard_normal((3, 6))
    mask = np.ones((3, 6))
    mask[:, 4:] = 0
    T2 = T.copy()
    T2[:, 4:] = 1e6
    l1, g1 = M.loss_and_grads(p, X, T, mask, shapes)
    l2, g2 = M.loss_and_grads(p, X, T2, mask, shapes)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_adam_first_step_is_signed_lr(M):
    """At t = 1 the bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8)
    assert np.abs(p + 0.01 * g / (np.abs(g) + 1e-8)).max() < 1e-15


def test_bf16_path_close_to_exact(M):
    rng = np.random.default_rng(3)
    shapes = M.layer_shapes()
    n = sum(o * i + o for o, i in shapes)
    p = rng.standard_normal(n) * 0.05
    X = rng.standard_normal((16, 4))
    Y, _ = M.forward(p, X, shapes)
    Yb, _ = M.forward(p, X, shapes, bf16=True)
    assert np.abs(Yb - Y).max() < 0.05 * np.abs(Y).max()
