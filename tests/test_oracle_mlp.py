"""Pins of the FP64 surrogate reference (oracle/mlp.py) to definitions independent of it:
the normal CDF by quadrature, a hand-worked network, finite-difference gradients, Adam's closed
form under a constant gradient, and envelope special cases."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import mlp


def _phi_quad(z):
    """Standard normal CDF by numerical integration of the density (independent of erf)."""
    val, _ = integrate.quad(lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi), -40.0, z, limit=200)
    return val


@pytest.mark.parametrize("z", [-3.0, -1.0, -0.2, 0.0, 0.5, 1.0, 2.5])
def test_gelu_is_z_times_normal_cdf(z):
    assert mlp.gelu(np.array(z)) == pytest.approx(z * _phi_quad(z), abs=1e-12)


def test_gelu_grad_matches_finite_differences():
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_hand_worked_network():
    """1 -> 1 -> 1: x = 1, W1 = 2, b1 = -1 -> z = 1, GELU(1) = Phi(1) = 0.8413447460685429;
    y = 3 GELU(1) + 0.5 = 3.0240342382056287 (Phi(1) from tables of the normal distribution)."""
    params = [(np.array([[2.0]]), np.array([-1.0])), (np.array([[3.0]]), np.array([0.5]))]
    Y, _ = mlp.forward(params, np.array([[1.0]]))
    assert Y[0, 0] == pytest.approx(3 * 0.8413447460685429 + 0.5, abs=1e-13)


def test_output_layer_is_affine_and_hidden_layers_are_not():
    """Scaling the input changes a hidden-only path non-linearly; the output bias shifts Y exactly."""
    params = mlp.init_params((5, 7, 3), seed=3)
    X = np.random.default_rng(1).standard_normal((4, 5))
    Y0, _ = mlp.forward(params, X)
    shifted = [params[0], (params[1][0], params[1][1] + np.array([1.0, -2.0, 0.5]))]
    Y1, _ = mlp.forward(shifted, X)
    np.testing.assert_allclose(Y1 - Y0, np.broadcast_to([1.0, -2.0, 0.5], Y0.shape), atol=1e-14)
    Y2, _ = mlp.forward(params, 2 * X)
    b = params[1][1]
    assert np.abs(Y2 - (2 * Y0 - b)).max() > 1e-3   # an affine map would give exactly 2 Y0 - b


def test_backward_matches_finite_differences():
    dims = (6, 9, 8, 5)
    params = mlp.init_params(dims, seed=11)
    params = [(W, b + 0.1 * np.arange(len(b))) for W, b in params]
    rng = np.random.default_rng(5)
    X = rng.standard_normal((7, dims[0]))
    T = rng.standard_normal((7, dims[-1]))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, mlp.loss_grad(Y, T))

    def L(p):
        return mlp.loss(mlp.forward(p, X)[0], T)

    h = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
                plus = [(W.copy(), b.copy()) for W, b in params]
                minus = [(W.copy(), b.copy()) for W, b in params]
                plus[li][which][idx] += h
                minus[li][which][idx] -= h
                fd = (L(plus) - L(minus)) / (2 * h)
                assert grads[li][which][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (li, which, idx)


def test_loss_and_gradient_definition():
    Y = np.array([[1.0, 2.0], [3.0, 5.0]])
    T = np.array([[0.0, 2.0], [3.0, 1.0]])
    assert mlp.loss(Y, T) == pytest.approx((1 + 0 + 0 + 16) / 4)
    np.testing.assert_allclose(mlp.loss_grad(Y, T), [[0.5, 0.0], [0.0, 2.0]])


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so every step
    moves each weight by -lr g / (|g| + eps): after t steps w = w0 - t lr g / (|g| + eps)."""
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4e-3]]), np.array([-2.0]))]
    state = mlp.adam_init(params)
    lr, eps = 1e-2, 1e-8
    p = params
    for t in range(1, 26):
        p, state = mlp.adam_step(p, grads, state, t, lr, eps=eps)
    np.testing.assert_allclose(p[0][0], params[0][0] - 25 * lr * grads[0][0] / (np.abs(grads[0][0]) + eps),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(p[0][1], params[0][1] - 25 * lr * grads[0][1] / (np.abs(grads[0][1]) + eps),
                               rtol=0, atol=1e-12)


def test_adam_first_moments_follow_the_recursion():
    """Two different gradients: m_2 = b1 (1-b1) g1 + (1-b1) g2, v_2 likewise with squares."""
    params = [(np.array([[0.0]]), np.array([0.0]))]
    s = mlp.adam_init(params)
    g1, g2 = 0.7, -0.2
    p, s = mlp.adam_step(params, [(np.array([[g1]]), np.array([0.0]))], s, 1, 1e-3)
    p, s = mlp.adam_step(p, [(np.array([[g2]]), np.array([0.0]))], s, 2, 1e-3)
    m, v = s[0][0][0, 0], s[0][1][0, 0]
    assert m == pytest.approx(0.9 * 0.1 * g1 + 0.1 * g2, rel=1e-14)
    assert v == pytest.approx(0.999 * 0.001 * g1 * g1 + 0.001 * g2 * g2, rel=1e-14)


def test_envelope_mask_cases():
    lo, hi = np.array([-1.0, -2.0, 0.0]), np.array([1.0, 2.0, 3.0])
    Xn = np.array([[0, 0, 1], [1, 2, 3], [-1, -2, 0], [1.0001, 0, 1], [0, 0, -1e-9], [np.nan, 0, 1]])
    # the box is closed; a non-finite feature is outside
    np.testing.assert_array_equal(mlp.envelope_mask(Xn, lo, hi), [0, 0, 0, 1, 1, 1])


def test_normalization_round_trip():
    X = np.random.default_rng(3).standard_normal((50, 4)) * [1, 10, 1e-4, 3] + [0, 5, 2e-4, -7]
    mu, sd = mlp.column_stats(X)
    Xn = mlp.normalize(X, mu, sd)
    np.testing.assert_allclose(Xn.mean(axis=0), 0, atol=1e-12)
    np.testing.assert_allclose(Xn.std(axis=0), 1, atol=1e-12)
