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


def test_round_bf16_matches_torch_and_ties_to_even():
    torch = __import__("pytest").importorskip("torch")
    g = starfield.rng(21)
    v = np.concatenate([g.normal(0, 1, 4000) * 10.0 ** g.integers(-6, 7, 4000), [0.0, -0.0, 1.0, -3.5]])
    v32 = v.astype(np.float32)
    ours = cnn.round_bf16(v32.astype(np.float64))
    theirs = torch.from_numpy(v32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(ours, theirs)
    # exact midpoints: BF16 spacing at 1 is 2^-7; ties go to the even significand
    assert cnn.round_bf16(1 + 2.0 ** -8) == 1.0
    assert cnn.round_bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert cnn.round_bf16(-(1 + 3 * 2.0 ** -8)) == -(1 + 2.0 ** -6)
    assert cnn.round_bf16(1 + 2.0 ** -8 + 2.0 ** -30) == 1 + 2.0 ** -7
    assert cnn.round_bf16(3.0 * 2.0 ** -100) == 3.0 * 2.0 ** -100


def test_bf16_storage_rounds_input_and_activations():
    n_out = 4
    params = starfield.cnn_init_params(n_out, 5).astype(np.float64)
    x, _ = _batch(2, n_out, 6)
    r = cnn.round_bf16
    a, _ = cnn.forward(params, x, n_out, rounding=r)
    b, _ = cnn.forward(params, r(x), n_out, rounding=r)
    np.testing.assert_array_equal(a, b)  # the input is rounded first
    assert np.abs(a - cnn.forward(params, x, n_out)[0]).max() > 0
    # closed form: zero conv weights, positive biases -> every stored activation is the
    # rounded bias chain, out = fc.w @ round(relu(b4)) + fc.b
    shapes = starfield.cnn_param_shapes(n_out)
    arrs = [np.zeros(s) for s in shapes]
    arrs[7] = np.linspace(0.1, 3.2, 32)
    arrs[8] = starfield.rng(2).normal(0, 1, (n_out, 32))
    arrs[9] = np.linspace(-1, 1, n_out)
    out, _ = cnn.forward(cnn.flatten(arrs), x, n_out, rounding=r)
    np.testing.assert_allclose(out, np.tile(arrs[8] @ r(arrs[7]) + arrs[9], (2, 1)), rtol=1e-13)
    assert np.abs(r(arrs[7]) - arrs[7]).max() > 1e-4


def test_bf16_storage_gradient_matches_torch_autograd():
    # the network with BF16 storage written with torch's conv2d and autograd: stored
    # values rounded on the way forward (identity derivative), the gradient at each
    # pre-activation rounded on the way back
    torch = __import__("pytest").importorskip("torch")
    F = torch.nn.functional
    r = cnn.round_bf16

    class StoreRound(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            return torch.from_numpy(r(a.detach().numpy()))

        @staticmethod
        def backward(ctx, g):
            return g

    class GradRound(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            return a.clone()

        @staticmethod
        def backward(ctx, g):
            return torch.from_numpy(r(g.detach().numpy()))

    n_out = 6
    params = starfield.cnn_init_params(n_out, 13).astype(np.float64)
    x, t = _batch(3, n_out, 14)
    loss_o, grad_o = cnn.loss_and_grad(params, x, t, n_out, rounding=r)
    ps = [torch.tensor(a, requires_grad=True) for a in cnn.unflatten(params, n_out)]
    h = StoreRound.apply(torch.from_numpy(x))
    for li, (_, stride) in enumerate(starfield.CNN_LAYERS):
        z = F.conv2d(h, ps[2 * li], ps[2 * li + 1], stride=stride, padding=1)
        h = StoreRound.apply(torch.relu(GradRound.apply(z)))
    out = h.mean(dim=(2, 3)) @ ps[-2].T + ps[-1]
    loss = ((out - torch.from_numpy(t)) ** 2).mean()
    loss.backward()
    grad_t = np.concatenate([p.grad.numpy().reshape(-1) for p in ps])
    assert abs(loss.item() - loss_o) <= 1e-12 * loss_o
    o = 0
    for shp in starfield.cnn_param_shapes(n_out):
        n = int(np.prod(shp))
        a, b = grad_o[o:o + n], grad_t[o:o + n]
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), shp
        o += n
