"""Pins of the FP64 conv-net oracle: the 3 x 3 convolution against scipy's library
correlate, and every gradient against central finite differences of the loss."""
import numpy as np
import pytest
import scipy.signal

from oracle import convnet as CN


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = CN.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate(x[n, :, :, c], W[o, :, :, c], mode="same") for c in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def _tiny(seed=1, channels=4, blocks=2, levels=3, H=5, Wd=6, N=2):
    rng = np.random.default_rng(seed)
    shapes = CN.layer_shapes(channels, blocks, levels)
    theta = np.concatenate([np.concatenate([0.4 * rng.standard_normal(co * 9 * ci), 0.1 * rng.standard_normal(co)])
                            for co, ci in shapes])
    inp = CN.net_input(rng.standard_normal((N, H, Wd)), rng.uniform(-3, -1, N))
    target = rng.standard_normal((N, H, Wd, levels))
    return shapes, theta, inp, target


def test_gradients_match_finite_differences():
    shapes, theta, inp, target = _tiny()
    loss, grads = CN.loss_and_grad(CN.unflatten(theta, shapes), inp, target)
    g = CN.flatten(grads)
    rng = np.random.default_rng(7)
    idx = rng.choice(theta.size, 60, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp = np.mean((CN.forward(CN.unflatten(tp, shapes), inp) - target) ** 2)
        lm = np.mean((CN.forward(CN.unflatten(tm, shapes), inp) - target) ** 2)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_conv_backward_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 4, 5, 2))
    W = rng.standard_normal((3, 3, 3, 2))
    dy = rng.standard_normal((1, 4, 5, 3))
    dx, dW, db = CN.conv3x3_backward(x, W, dy)
    eps = 1e-6
    for i in range(x.size):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[i] += eps
        xm[i] -= eps
        f = lambda v: float(np.sum(dy * CN.conv3x3(v.reshape(x.shape), W, np.zeros(3))))
        assert abs((f(xp) - f(xm)) / (2 * eps) - dx.ravel()[i]) < 1e-6


def test_zero_head_gives_zero_correction():
    # with the head's weights and bias at zero the network predicts u^n - u^0 = 0: the plain guess
    shapes, theta, inp, target = _tiny(levels=3)
    params = CN.unflatten(theta, shapes)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros_like(params[-1][1]))
    assert np.all(CN.forward(params, inp) == 0.0)
