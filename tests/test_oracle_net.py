"""Pins of the FP64 network oracle: closed forms of the convolution and central
finite differences of the loss (none retypes the oracle's formulas)."""
import numpy as np
import pytest

from oracle import net

RNG = np.random.default_rng(7)


def test_conv_identity_and_shift_kernels():
    x = RNG.normal(size=(5, 6, 7, 2))
    W = np.zeros((27, 2, 2))
    W[13] = np.eye(2)  # centre tap
    np.testing.assert_array_equal(net.conv(x, W), x)
    W = np.zeros((27, 2, 2))
    t = net.TAPS.index((0, 0, 1))
    W[t] = np.eye(2)  # reads x[.., x+1]: output is x shifted left, zero at the end
    y = net.conv(x, W)
    np.testing.assert_array_equal(y[:, :, :-1], x[:, :, 1:])
    assert np.all(y[:, :, -1] == 0)


def test_conv_box_filter_sums_neighbourhood():
    x = RNG.normal(size=(6, 5, 4, 1))
    W = np.ones((27, 1, 1))
    y = net.conv(x, W)
    # brute force: 3x3x3 sum with zero padding
    p = np.pad(x[..., 0], 1)
    ref = sum(p[1 + dz:7 + dz, 1 + dy:6 + dy, 1 + dx:5 + dx] for dz, dy, dx in net.TAPS)
    np.testing.assert_allclose(y[..., 0], ref, atol=1e-12)


def test_conv_gradients_are_adjoint():
    x = RNG.normal(size=(4, 5, 6, 3))
    W = RNG.normal(size=(27, 3, 2))
    dy = RNG.normal(size=(4, 5, 6, 2))
    dx, dW = net.conv_grads(x, W, dy)
    # <conv(x, W), dy> is bilinear: its gradients reproduce it exactly
    s = np.sum(net.conv(x, W) * dy)
    assert np.sum(dx * x) == pytest.approx(s, rel=1e-12)
    assert np.sum(dW * W) == pytest.approx(s, rel=1e-12)


def _weights(C=4, seed=3):
    r = np.random.default_rng(seed)
    return (r.normal(size=(27, 1, C)) * 0.3, r.normal(size=(27, C, C)) * 0.2, r.normal(size=(27, C, 1)) * 0.3)


@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 7, 8)])
def test_loss_gradient_matches_central_differences(shape):
    Ws = _weights()
    x = RNG.normal(size=shape)
    t = RNG.normal(size=shape)
    L, dWs, _ = net.backward(x, Ws, t)
    h = 1e-6
    for k in range(3):
        for _ in range(6):
            idx = tuple(RNG.integers(0, s) for s in Ws[k].shape)
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[k][idx] += h
            Wm[k][idx] -= h
            fd = (net.loss(net.forward(x, Wp)[0], t) - net.loss(net.forward(x, Wm)[0], t)) / (2 * h)
            assert dWs[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_network_is_positively_homogeneous():
    # bias-free ReLU net: scaling the input scales the output (like A^-1)
    Ws = _weights()
    x = RNG.normal(size=(3, 4, 5))
    y1 = net.forward(x, Ws)[0]
    y2 = net.forward(3.7 * x, Ws)[0]
    np.testing.assert_allclose(y2, 3.7 * y1, rtol=1e-12, atol=1e-14)


def test_backward_loss_of_an_identity_network_is_its_closed_form():
    # centre-tap identity weights pass a positive input through both ReLUs
    # unchanged, so y = x and the relative loss is |x - t|^2 / |t|^2 exactly:
    # 1/4 for t = 2x, 4 for t = -x
    x = np.abs(RNG.normal(size=(4, 5, 6))) + 0.1
    W1, W2, W3 = np.zeros((27, 1, 3)), np.zeros((27, 3, 3)), np.zeros((27, 3, 1))
    W1[13, 0, 0] = W2[13, 0, 0] = W3[13, 0, 0] = 1.0
    Ws = (W1, W2, W3)
    y, _ = net.forward(x, Ws)
    np.testing.assert_array_equal(y, x)
    for t, want in ((2.0 * x, 0.25), (-x, 4.0)):
        L, _, _ = net.backward(x, Ws, t)
        assert L == pytest.approx(want, rel=1e-14)
        assert net.loss(y, t) == pytest.approx(want, rel=1e-14)
