"""Pins of the FP64 coefficient-network oracle (CPU): finite differences of the loss and
scipy's correlation for the convolution layers."""
import numpy as np
import scipy.signal

import starfield
from oracle import cnn


def _batch(B, n_out, seed):
    g = starfield.rng(seed)
    x = g.normal(0, 1, (B, 2, starfield.CNN_IN, starfield.CNN_IN))
    t = g.normal(0, 1, (B, n_out))
    return x, t


def test_conv_forward_matches_scipy_correlate():
    g = starfield.rng(1)
    x = g.normal(0, 1, (2, 3, 9, 10))
    w = g.normal(0, 1, (4, 3, 3, 3))
    b = g.normal(0, 1, 4)
    for stride in (1, 2):
        out = cnn.conv_fwd(x, w, b, stride)
        for bi in range(2):
            for o in range(4):
                ref = sum(scipy.signal.correlate2d(x[bi, c], w[o, c], mode="same") for c in range(3)) + b[o]
                np.testing.assert_allclose(out[bi, o], ref[::stride, ::stride], rtol=1e-12, atol=1e-12)


def test_param_count():
    n = sum(int(np.prod(s)) for s in starfield.cnn_param_shapes(49))
    assert n == (32 * 2 * 9 + 32) + 3 * (32 * 32 * 9 + 32) + 49 * 32 + 49
    assert starfield.cnn_init_params(49, 3).size == n


def test_gradient_matches_finite_differences():
    n_out = 5
    params = starfield.cnn_init_params(n_out, 7).astype(np.float64)
    x, t = _batch(2, n_out, 8)
    loss, grad = cnn.loss_and_grad(params, x, t, n_out)
    g = starfield.rng(9)
    idx = g.choice(params.size, 40, replace=False)
    # include biases and the linear layer explicitly
    idx = np.concatenate([idx, [32 * 2 * 9, params.size - 1, params.size - n_out - 3]])
    eps = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (cnn.loss_and_grad(pp, x, t, n_out)[0] - cnn.loss_and_grad(pm, x, t, n_out)[0]) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_linear_output_layer_closed_form():
    # with all conv weights zero and positive conv biases, every activation equals the bias
    # chain, so the output is fc.w @ relu(b4) + fc.b exactly
    n_out = 3
    shapes = starfield.cnn_param_shapes(n_out)
    arrs = [np.zeros(s) for s in shapes]
    arrs[7] = np.linspace(0.1, 3.2, 32)  # conv4 bias
    arrs[8] = starfield.rng(2).normal(0, 1, (n_out, 32))
    arrs[9] = np.array([0.5, -1.0, 2.0])
    params = cnn.flatten(arrs)
    x, _ = _batch(2, n_out, 3)
    out, _ = cnn.forward(params, x, n_out)
    np.testing.assert_allclose(out, np.tile(arrs[8] @ arrs[7] + arrs[9], (2, 1)), rtol=1e-13)
