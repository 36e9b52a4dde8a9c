"""The coefficient network on the device: forward and gradients against the FP64 oracle
(same BF16-rounded weights), the optimiser step, the polynomial field fit, and training on
pairs the plain method generates (loss falls, predictions beat the prior, the network path
is faster than the FP64 fit, and the fallback hands bad predictions to the fit)."""
import time

import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
import starfield
from oracle import cnn as ocnn
from paper_1209_5823_gb300 import learned

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _data(B, n_out, seed):
    g = starfield.rng(seed)
    x = g.normal(0, 1, (B, 2, 64, 64)).astype(np.float32)
    t = g.normal(0, 1, (B, n_out)).astype(np.float32)
    return x, t


# The network stores its input, activations and pre-activation gradients in BF16 and
# sums in FP32; the oracle rounds the same values (FP64 otherwise).  What remains are
# FP32 summation errors and rare rounding flips, where the two sides' unrounded values
# straddle a BF16 rounding boundary (or a ReLU's zero) and a stored value differs by one
# BF16 step.  Bars: outputs within 1e-3 of their largest value (measured <= 2.5e-4 up to
# 256 stamps), each gradient block within one BF16 step, 2^-8, of its largest value
# (measured <= 1.6e-3); against the plain FP64 network the gradients differ by up to 16 %.
TOL_OUT = 1e-3
TOL_GRAD = 2.0 ** -8


def _check_against_oracle(B, n_out, seed):
    p = starfield.cnn_init_params(n_out, seed)
    x, t = _data(B, n_out, seed + 1)
    dp, dx, dt = (torch.from_numpy(a).cuda() for a in (p, x, t))
    out = svk.svk_cnn_forward(dp, dx, n_out).cpu().numpy()
    grad, loss = svk.svk_cnn_gradient(dp, dx, dt)
    assert svk.svk_device_status() == svk.SVK_OK
    pq = bf16_round(p).astype(np.float64)
    ref_out, _ = ocnn.forward(pq, x.astype(np.float64), n_out, rounding=ocnn.round_bf16)
    ref_loss, ref_grad = ocnn.loss_and_grad(pq, x.astype(np.float64), t.astype(np.float64), n_out,
                                            rounding=ocnn.round_bf16)
    assert np.abs(out - ref_out).max() <= TOL_OUT * np.abs(ref_out).max()
    assert abs(float(loss.item()) - ref_loss) <= TOL_OUT * ref_loss
    g = grad.cpu().numpy().astype(np.float64)
    # every parameter block separately (scales differ by orders of magnitude)
    o = 0
    for shp in starfield.cnn_param_shapes(n_out):
        n = int(np.prod(shp))
        a, b = g[o:o + n], ref_grad[o:o + n]
        assert np.abs(a - b).max() <= TOL_GRAD * np.abs(b).max() + 1e-9, shp
        o += n


@pytest.mark.parametrize("n_out", [49, 7])
def test_forward_and_gradient_match_oracle(n_out):
    _check_against_oracle(3, n_out, 11)


def test_ragged_batch_matches_oracle():
    # 37 stamps: the 8x8 layers end in a partial 128-row tile, and the first layer's last
    # weight-gradient chunk is shorter than the others
    _check_against_oracle(37, 49, 21)


def test_training_batch_matches_oracle():
    # the training batch (256 stamps): the weight gradients are split into the chunk
    # counts and reduced in the fixed order that training runs
    _check_against_oracle(256, 49, 31)


def test_forward_4096_sampled_matches_oracle():
    # the 4096-stamp forward pass the bench times; each stamp's output depends on that
    # stamp alone, so 64 seeded stamps of it are compared with the oracle
    n_out, B = 49, 4096
    p = starfield.cnn_init_params(n_out, 41)
    x, _ = _data(B, n_out, 42)
    out = svk.svk_cnn_forward(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(), n_out).cpu().numpy()
    assert svk.svk_device_status() == svk.SVK_OK
    pick = np.sort(starfield.rng(43).choice(B, 64, replace=False))
    pick[-1] = B - 1  # the last tile of every layer included
    ref, _ = ocnn.forward(bf16_round(p).astype(np.float64), x[pick].astype(np.float64), n_out,
                          rounding=ocnn.round_bf16)
    assert np.abs(out[pick] - ref).max() <= TOL_OUT * np.abs(ref).max()


def test_gradient_is_deterministic():
    n_out = 49
    p = torch.from_numpy(starfield.cnn_init_params(n_out, 3)).cuda()
    x, t = (torch.from_numpy(a).cuda() for a in _data(300, n_out, 4))
    g1, _ = svk.svk_cnn_gradient(p, x, t)
    g2, _ = svk.svk_cnn_gradient(p, x, t)
    assert torch.equal(g1, g2)


def test_gradient_calls_from_two_threads():
    # the weight gradients run on a library stream forked from and joined back into the
    # caller's stream; two host threads on their own streams (and workspaces) must each get
    # exactly the single-threaded result while their calls interleave
    import threading
    n_out, B = 49, 256
    p = torch.from_numpy(starfield.cnn_init_params(n_out, 5)).cuda()
    data = [tuple(torch.from_numpy(a).cuda() for a in _data(B, n_out, 40 + i)) for i in range(2)]
    ref = [svk.svk_cnn_gradient(p, x, t)[0].clone() for x, t in data]
    torch.cuda.synchronize()
    nbytes = svk.svk_cnn_workspace_size(B, n_out)
    out = [[], []]
    errors = []

    def worker(i):
        try:
            s = torch.cuda.Stream()
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            x, t = data[i]
            with torch.cuda.stream(s):
                for _ in range(20):
                    g = torch.empty_like(p)
                    svk.svk_cnn_gradient(p, x, t, grad=g, workspace=ws, stream=s)
                    out[i].append(g)
            s.synchronize()
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    assert not errors, errors
    for i in range(2):
        assert len(out[i]) == 20
        for g in out[i]:
            assert torch.equal(g, ref[i])


def test_adam_step():
    n = 1000
    g = starfield.rng(3)
    p = g.normal(0, 1, n).astype(np.float32)
    gr = g.normal(0, 1, n).astype(np.float32)
    dp, dm, dv, dg = (torch.from_numpy(a).cuda() for a in (p.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32), gr))
    svk.svk_cnn_adam(dp, dm, dv, dg, 1, lr=0.01)
    # first bias-corrected Adam step is lr * g / (|g| + eps)
    exp = p - 0.01 * gr / (np.abs(gr) + 1e-8)
    np.testing.assert_allclose(dp.cpu().numpy(), exp, rtol=0, atol=1e-6)


def test_field_fit_recovers_polynomial():
    W, H, d, N, S = 4096, 2048, 2, 5, 200
    g = starfield.rng(4)
    xy = np.stack([g.integers(0, W, S), g.integers(0, H, S)], 1).astype(np.int32)
    c = g.normal(0, 1, (N, 6))
    xt = (2 * xy[:, 0] - (W - 1)) / (W - 1)
    yt = (2 * xy[:, 1] - (H - 1)) / (H - 1)
    mono = np.stack([np.ones(S), yt, yt ** 2, xt, xt * yt, xt ** 2], 1)
    local = (mono @ c.T).astype(np.float32)
    co, info = svk.svk_cnn_field_fit(torch.from_numpy(local).cuda(), torch.from_numpy(xy).cuda(), W, H, d)
    assert int(info.item()) == -1
    np.testing.assert_allclose(co.cpu().numpy(), c, rtol=0, atol=2e-5)


@pytest.mark.parametrize("S,N,d,weighted", [(700, 49, 3, True), (257, 49, 2, False), (1, 3, 0, False),
                                              (600, 130, 1, True)])
def test_field_fit_matches_weighted_least_squares(S, N, d, weighted):
    # several stamp chunks and coefficient blocks; weighted normal equations against
    # numpy's least squares on sqrt(w)-scaled rows (FP64)
    W, H = 2048, 4096
    g = starfield.rng(40 + S + N)
    xy = np.stack([g.integers(0, W, S), g.integers(0, H, S)], 1).astype(np.int32)
    xt = (2.0 * xy[:, 0] - (W - 1)) / (W - 1)
    yt = (2.0 * xy[:, 1] - (H - 1)) / (H - 1)
    mono = np.stack([xt ** p * yt ** q for p in range(d + 1) for q in range(d + 1 - p)], 1)
    local = g.normal(0, 1, (S, N)).astype(np.float32)
    w = g.uniform(0.5, 2.0, S).astype(np.float32) if weighted else np.ones(S, np.float32)
    co, info = svk.svk_cnn_field_fit(torch.from_numpy(local).cuda(), torch.from_numpy(xy).cuda(), W, H, d,
                                     weights=torch.from_numpy(w).cuda() if weighted else None)
    assert int(info.item()) == -1
    sw = np.sqrt(w.astype(np.float64))[:, None]
    ref = np.linalg.lstsq(mono * sw, local.astype(np.float64) * sw, rcond=None)[0].T  # [N][T]
    np.testing.assert_allclose(co.cpu().numpy(), ref, rtol=0, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_field_fit_reports_a_singular_system():
    # every stamp at the frame centre (xt = yt = 0): only the constant term is determined
    xy = np.tile(np.array([[500, 500]], np.int32), (50, 1))
    local = np.ones((50, 7), np.float32)
    co, info = svk.svk_cnn_field_fit(torch.from_numpy(local).cuda(), torch.from_numpy(xy).cuda(), 1001, 1001, 2)
    assert int(info.item()) >= 0
    assert not co.abs().sum().item()


def _field(W, H, seed):
    g = starfield.rng(seed)
    cat = starfield.star_catalog(W, H, int(W * H * 0.0024), g)
    R = starfield.add_noise(starfield.render(cat, W, H), 30.0, g).astype(np.float32)
    return torch.from_numpy(R).cuda(), cat


def test_training_learns_and_network_path_is_faster_with_fallback():
    dev = torch.device("cuda")
    L, N = 19, 49
    basis = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    prior = learned.CoeffPrior(N)
    gen = torch.Generator(device="cuda").manual_seed(5)
    Rf, cat = _field(1024, 1024, 6)
    bright = np.argsort(cat.flux)[::-1][:3000]
    cx = torch.from_numpy(np.clip(cat.x[bright].astype(np.int64), 48, 1024 - 48)).cuda()
    cy = torch.from_numpy(np.clip(cat.y[bright].astype(np.int64), 48, 1024 - 48)).cuda()
    n = cx.numel()
    a = prior.mean(dev) + prior.std(dev) * torch.randn((n, N), device=dev, generator=gen)
    x, _, _ = learned.make_pairs(Rf, cx, cy, a, basis, 30.0, gen)
    ntr = n - 500
    net = learned.CoefficientNetwork(torch.from_numpy(starfield.cnn_init_params(N, 7)).cuda(), prior, batch=128,
                                     seed=5)
    losses = net.train(x[:ntr], a[:ntr], 800, lr=3e-3).cpu().numpy()
    assert losses[-50:].mean() < 0.92 * losses[:50].mean()
    pred = net.predict(x[ntr:])
    err_net = float(((pred - a[ntr:]) / prior.std(dev)).pow(2).mean())
    # predicting the prior mean scores 1.0 (+- 0.01 over 500 x 49 held-out values)
    assert err_net < 0.95

    # a frame whose kernel has spatially varying coefficients: network path vs FP64 fit, both
    # for the cubic 49 x 10 field (the fit's moments grow with the degree, the network's
    # cost does not; with few stamps the fit can be the faster one)
    W = H = 1024
    D = 3
    c_true = torch.from_numpy(starfield.planted_coeffs(N, D, starfield.rng(8)).astype(np.float32)).cuda()
    I = svk.svk_convolve(Rf, basis, c_true, D, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    I = I + 30.0 * torch.randn(I.shape, device=dev, generator=gen)
    st = torch.stack([cx[:300], cy[:300]], 1).to(torch.int32)
    learned.apply_to_frame(net, Rf, I, st, basis, D, 30.0, fallback_ratio=1e9, reference_noise_sigma=0.0)  # warm both paths
    svk.svk_fit_coeffs(Rf, I, st, 41, basis, D, bg_degree=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = learned.apply_to_frame(net, Rf, I, st, basis, D, 30.0, fallback_ratio=1e9, reference_noise_sigma=0.0)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    t0 = time.perf_counter()
    svk.svk_fit_coeffs(Rf, I, st, 41, basis, D, bg_degree=0)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    assert res["source"] == "network" and t_net < t_fit
    # garbage weights: the residual check hands the frame to the fit
    bad = learned.CoefficientNetwork(torch.zeros_like(net.params), learned.CoeffPrior(N, mean0=0.0), batch=128)
    res2 = learned.apply_to_frame(bad, Rf, I, st, basis, D, 30.0, fallback_ratio=2.0, reference_noise_sigma=0.0)
    assert res2["source"] == "fit"


def test_training_checkpoint_resumes_bit_exactly(tmp_path):
    # weights, Adam moments, step and the batch-draw seed saved mid-run (the draws are fixed
    # by seed and step): the resumed run ends with the same weights, bit for bit, as an
    # uninterrupted one; 20 steps = two 8-step graphs and four single steps, 8 + 12 splits
    # them differently
    N = 49
    g0 = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn((600, 2, 64, 64), device="cuda", generator=g0) * 0.3
    a = torch.randn((600, N), device="cuda", generator=g0) * 0.02 + learned.CoeffPrior(N).mean(torch.device("cuda"))
    init = torch.from_numpy(starfield.cnn_init_params(N, 3)).cuda()

    full = learned.CoefficientNetwork(init.clone(), learned.CoeffPrior(N), batch=64, seed=12)
    lf = full.train(x, a, 20, lr=2e-3)

    part = learned.CoefficientNetwork(init.clone(), learned.CoeffPrior(N), batch=64, seed=12)
    lp = part.train(x, a, 8, lr=2e-3)
    torch.save({"net": part.state_dict()}, tmp_path / "ckpt.pt")
    del part

    ck = torch.load(tmp_path / "ckpt.pt")
    resumed = learned.CoefficientNetwork.from_state_dict(ck["net"], device="cuda")
    lr_ = resumed.train(x, a, 12, lr=2e-3)
    assert resumed.step == full.step == 20
    assert torch.equal(resumed.params, full.params)
    assert torch.equal(resumed.m, full.m) and torch.equal(resumed.v, full.v)
    # the same losses step by step (the loss value itself is summed with float atomics, so
    # to its last bits only)
    assert torch.allclose(torch.cat([lp, lr_]), lf, rtol=1e-6, atol=0)
    # another seed draws other batches
    other = learned.CoefficientNetwork(init.clone(), learned.CoeffPrior(N), batch=64, seed=13)
    other.train(x, a, 20, lr=2e-3)
    assert not torch.equal(other.params, full.params)


def test_adam_device_step_matches_host_step():
    # the step count read from device memory: the same update as svk_cnn_adam over several
    # steps (bias corrections formed on the device instead of the host: float32 rounding)
    n = 5000
    g = starfield.rng(31)
    p0 = g.normal(0, 1, n).astype(np.float32)
    grads = [g.normal(0, 1, n).astype(np.float32) for _ in range(5)]
    a = [torch.from_numpy(v).cuda() for v in (p0.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32))]
    b = [torch.from_numpy(v).cuda() for v in (p0.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32))]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for k, gr in enumerate(grads, start=1):
        dg = torch.from_numpy(gr).cuda()
        svk.svk_cnn_adam(a[0], a[1], a[2], dg, k, lr=0.01)
        step.fill_(k)
        svk.svk_cnn_adam_device_step(b[0], b[1], b[2], dg, step, lr=0.01)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        np.testing.assert_allclose(y.cpu().numpy(), x.cpu().numpy(), rtol=1e-5, atol=1e-6)
