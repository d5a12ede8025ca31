"""Pins of the oracle's learned-smoother network (no counterpart in the paper):
finite differences, adjointness and delta-kernel identities."""
import numpy as np
import pytest

from oracle import cnn


def _weights(C=4, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((C, 1, 3, 3)) * 0.5, rng.standard_normal((C, C, 3, 3)) * 0.3,
            rng.standard_normal((1, C, 3, 3)) * 0.3)


def test_delta_kernel_is_identity_and_shift():
    a = np.random.default_rng(1).standard_normal((2, 3, 7, 9))
    W = np.zeros((3, 3, 3, 3))
    for c in range(3):
        W[c, c, 1, 1] = 1.0
    assert np.array_equal(cnn.conv3x3(a, W), a)
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 1, 2] = 1.0                                     # reads the right neighbour
    out = cnn.conv3x3(a[:, :1], W)
    assert np.array_equal(out[..., :-1], a[:, :1, :, 1:]) and np.all(out[..., -1] == 0)


def test_convolution_adjoint_identity():
    rng = np.random.default_rng(2)
    a, g = rng.standard_normal((2, 3, 6, 5)), rng.standard_normal((2, 4, 6, 5))
    W = rng.standard_normal((4, 3, 3, 3))
    lhs = np.sum(cnn.conv3x3(a, W) * g)
    rhs = np.sum(a * cnn.conv3x3_adjoint(g, W))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the weight gradient is the derivative of the same bilinear form
    dW = cnn.conv3x3_weight_grad(a, g)
    assert abs(np.sum(dW * W) - lhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_loss_gradients_match_central_differences(layer):
    rng = np.random.default_rng(3)
    r, e = rng.standard_normal((2, 6, 7)), rng.standard_normal((2, 6, 7))
    Ws = list(_weights(seed=4))
    loss, grads = cnn.loss_and_grads(r, e, Ws)
    W = Ws[layer]
    idx = [tuple(rng.integers(0, s) for s in W.shape) for _ in range(6)]
    h = 1e-6
    for ix in idx:
        Wp = [w.copy() for w in Ws]
        Wm = [w.copy() for w in Ws]
        Wp[layer][ix] += h
        Wm[layer][ix] -= h
        fd = (cnn.loss_and_grads(r, e, Wp)[0] - cnn.loss_and_grads(r, e, Wm)[0]) / (2 * h)
        assert abs(fd - grads[layer][ix]) <= 1e-6 * max(1.0, abs(fd)), (layer, ix)


def test_network_is_positively_homogeneous():
    """No biases: CNN(alpha r) = alpha CNN(r) for alpha > 0 (what lets the solver
    apply it to unscaled residuals)."""
    r = np.random.default_rng(5).standard_normal((1, 8, 8))
    Ws = _weights(seed=6)
    y1, _ = cnn.forward(r, Ws)
    y2, _ = cnn.forward(3.7e-9 * r, Ws)
    assert np.allclose(y2, 3.7e-9 * y1, rtol=1e-12, atol=0)


def test_adam_first_step_moves_by_learning_rate():
    w, g = np.array([1.0, -2.0]), np.array([0.3, -4.0])
    w1, m, v = cnn.adam_step(w, g, np.zeros(2), np.zeros(2), 1, 0.01)
    assert np.allclose(w1, w - 0.01 * np.sign(g), atol=1e-7)
