"""Pins for the FP64 corrector oracle: its convolution against brute-force
loops, the adjoint identity of its transposed convolution, its whole-network
gradient against central finite differences, and the first Adam step against
the closed form lr * sign(g)."""
import numpy as np
import pytest

from oracle import corrector as oc
from paper_1706_02261_b300 import inputs


def brute_conv(X, W, b):
    Bn, C, H, Wd = X.shape
    O = W.shape[0]
    Y = np.zeros((Bn, O, H, Wd))
    for bb in range(Bn):
        for o in range(O):
            for y in range(H):
                for x in range(Wd):
                    acc = b[o]
                    for c in range(C):
                        for i in range(3):
                            for j in range(3):
                                acc += W[o, c, i, j] * X[bb, c, (y + i - 1) % H, (x + j - 1) % Wd]
                    Y[bb, o, y, x] = acc
    return Y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2, 3, 4, 5))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    assert np.allclose(oc.conv(X, W, b), brute_conv(X, W, b), atol=1e-12)


def test_conv_transpose_is_the_adjoint():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, 3, 6, 7))
    W = rng.standard_normal((5, 3, 3, 3))
    Y = rng.standard_normal((2, 5, 6, 7))
    lhs = np.sum(oc.conv(X, W, None) * Y)
    rhs = np.sum(X * oc.conv_transpose(Y, W))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("c_in", [2, 3])
def test_network_gradient_matches_finite_differences(c_in):
    rng = np.random.default_rng(2)
    theta = inputs.corrector_init(c_in, 3)
    # give the zero last layer and the biases some weight so every path is exercised
    theta += 0.05 * rng.standard_normal(theta.size)
    X = rng.standard_normal((2, c_in, 6, 5))
    T = rng.standard_normal((2, 2, 6, 5))
    sigma = 0.3
    loss, g = oc.loss_and_grad(theta, X, T, sigma)
    idx = rng.choice(theta.size, size=120, replace=False)
    h = 1e-6
    for k in idx:
        tp = theta.copy()
        tp[k] += h
        tm = theta.copy()
        tm[k] -= h
        fd = (oc.loss_and_grad(tp, X, T, sigma)[0] - oc.loss_and_grad(tm, X, T, sigma)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8, (k, fd, g[k])


def test_untrained_corrector_is_identity_and_count():
    theta = inputs.corrector_init(2, 0)
    assert theta.size == oc.param_count(2) == inputs.corrector_param_count(2)
    X = np.random.default_rng(4).standard_normal((1, 2, 8, 8))
    out, _, _ = oc.forward(theta, X)
    assert np.array_equal(out, X[:, :2])


def test_first_adam_step_moves_by_lr_sign_g():
    g = np.array([3.0, -0.2, 1e-3, -7.0])
    th, m, v = oc.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 1e-3)
    assert np.allclose(th, -1e-3 * np.sign(g), rtol=1e-4)


def test_bf16_rounding_of_the_inference_activations():
    """round_bf16: representable values stay, ties go to the even neighbour,
    and act_bf16=False leaves the forward pass unchanged."""
    one_ulp = 2.0 ** -7                                       # bfloat16 spacing on [1, 2)
    vals = np.array([1.0, 1.0 + one_ulp, 1.0 + one_ulp / 2, 1.0 + 3 * one_ulp / 2, -2.5, 0.0])
    got = oc.round_bf16(vals)
    assert np.array_equal(got, [1.0, 1.0 + one_ulp, 1.0, 1.0 + 2 * one_ulp, -2.5, 0.0])
    rng = np.random.default_rng(9)
    theta = rng.standard_normal(oc.param_count(2)) * 0.1
    X = rng.standard_normal((1, 2, 8, 8))
    a, _, _ = oc.forward(theta, X, 0.5)
    b, _, _ = oc.forward(theta, X, 0.5, act_bf16=False)
    c, _, _ = oc.forward(theta, X, 0.5, act_bf16=True)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
