"""The data side of the coefficient network through the C ABI: stamps and their
normalisation, target standardisation, the residual check that keeps or rejects the
network's coefficients (with its decision pinned on constructed residuals), and the
device-side pieces of a training step (batch draw, row gather, step bookkeeping)."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
import starfield

pytestmark = pytest.mark.gpu


def _padded(a, extra):
    """a float32 [H][W] copied into the first W columns of a [H][W + extra] device buffer."""
    H, W = a.shape
    buf = torch.full((H, W + extra), float("nan"), dtype=torch.float32, device="cuda")
    buf[:, :W] = torch.from_numpy(a).cuda()
    return buf[:, :W]


def _ref_stamps(img, xy, size, offset, divisor):
    H, W = img.shape
    half = size // 2
    out = np.zeros((len(xy), size, size), np.float32)
    for s, (cx, cy) in enumerate(xy):
        for v in range(size):
            for u in range(size):
                x, y = cx - half + u, cy - half + v
                val = img[y, x] if (0 <= x < W and 0 <= y < H) else np.float32(0)
                out[s, v, u] = np.float32(val - np.float32(offset)) / np.float32(divisor)
    return out


def test_cut_stamps_matches_reference_and_fills_channels():
    g = starfield.rng(201)
    img = (1000 + 300 * g.standard_normal((200, 300))).astype(np.float32)
    # centres inside, on the edges and beyond them (zero counts outside the frame)
    xy = np.array([[150, 100], [0, 0], [299, 199], [-3, 50], [310, 205], [5, 190]], np.int32)
    dimg = _padded(img, 29)
    got = svk.svk_cut_stamps(dimg, torch.from_numpy(xy).cuda(), 16, 1000.0, 3000.0).cpu().numpy()
    np.testing.assert_array_equal(got, _ref_stamps(img, xy, 16, 1000.0, 3000.0))
    # two images into the channels of one [n][2][S][S] input
    img2 = (img * 0.5 + 7).astype(np.float32)
    x = torch.full((len(xy), 2, 16, 16), float("nan"), device="cuda")
    svk.svk_cut_stamps(dimg, torch.from_numpy(xy).cuda(), 16, 1000.0, 3000.0, out=x, stamp_stride=512)
    svk.svk_cut_stamps(torch.from_numpy(img2).cuda(), torch.from_numpy(xy).cuda(), 16, 1000.0, 3000.0, out=x[:, 1],
                       stamp_stride=512)
    np.testing.assert_array_equal(x[:, 0].cpu().numpy(), _ref_stamps(img, xy, 16, 1000.0, 3000.0))
    np.testing.assert_array_equal(x[:, 1].cpu().numpy(), _ref_stamps(img2, xy, 16, 1000.0, 3000.0))
    with pytest.raises(svk.SvkError):
        svk.svk_cut_stamps(dimg, torch.from_numpy(xy).cuda(), 16, 0.0, 0.0)


def _ref_residual(D, xy, size):
    H, W = D.shape
    half = size // 2
    tot = 0.0
    for cx, cy in xy:
        st = np.zeros((size, size))
        for v in range(size):
            for u in range(size):
                x, y = cx - half + u, cy - half + v
                if 0 <= x < W and 0 <= y < H:
                    st[v, u] = D[y, x]
        tot += ((st - st.mean()) ** 2).sum()
    return tot / (len(xy) * size * size)


def test_stamp_residual_value_and_decision():
    g = starfield.rng(202)
    H, W, size, sig = 256, 320, 21, 30.0
    xy = np.stack([g.integers(0, W, 40), g.integers(0, H, 40)], 1).astype(np.int32)  # some cross the edges
    K0 = np.zeros((11, 11), np.float32)
    K0[5, 5] = 0.6
    K0[5, 4] = K0[4, 5] = 0.2
    k0 = torch.from_numpy(K0).cuda()
    dxy = torch.from_numpy(xy).cuda()
    floor = sig ** 2 + 10.0 ** 2 * float((K0.astype(np.float64) ** 2).sum())
    for scale, expect in ((1.0, 0), (3.0, 1)):
        D = (scale * sig * g.standard_normal((H, W)) + 17.0).astype(np.float32)  # an offset the stamp means remove
        out, fb = svk.svk_stamp_residual(_padded(D, 5), dxy, size, k0, sig, 10.0, 2.0)
        chi2, fl = out.cpu().numpy()
        assert abs(chi2 - _ref_residual(D.astype(np.float64), xy, size)) <= 1e-12 * chi2
        assert abs(fl - floor) <= 1e-12 * floor
        assert int(fb.item()) == expect  # 1 sigma: kept; 3 sigma: above twice the floor, handed to the fit
    # a failed field fit hands the frame to the fit whatever the residual
    D = (sig * g.standard_normal((H, W))).astype(np.float32)
    for info, expect in ((-1, 0), (0, 1), (7, 1)):
        fi = torch.tensor([info], dtype=torch.int32, device="cuda")
        _, fb = svk.svk_stamp_residual(_padded(D, 0), dxy, size, k0, sig, 10.0, 2.0, field_info=fi)
        assert int(fb.item()) == expect
    # deterministic: the same sums in the same order
    a, _ = svk.svk_stamp_residual(_padded(D, 0), dxy, size, k0, sig, 10.0, 2.0)
    b, _ = svk.svk_stamp_residual(_padded(D, 0), dxy, size, k0, sig, 10.0, 2.0)
    assert torch.equal(a, b)


def test_standardise_round_trip():
    g = starfield.rng(203)
    a = (g.standard_normal((300, 49)) * 0.02).astype(np.float32)
    a[:, 0] += 1.0
    mean = np.zeros(49, np.float32)
    mean[0] = 1.0
    sd = np.full(49, 0.02, np.float32)
    sd[0] = 0.03
    dm, ds = torch.from_numpy(mean).cuda(), torch.from_numpy(sd).cuda()
    z = svk.svk_cnn_standardise(torch.from_numpy(a).cuda(), dm, ds)
    np.testing.assert_array_equal(z.cpu().numpy(), (a - mean) / sd)  # IEEE float32 subtract and divide
    back = svk.svk_cnn_standardise(z, dm, ds, inverse=True).cpu().numpy()
    np.testing.assert_allclose(back, a, rtol=0, atol=1e-7)


def _splitmix64(z):
    """SplitMix64 output function for counter z (Steele, Lea and Flood, OOPSLA 2014)."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_draw_batch_follows_its_definition_and_is_uniform():
    seed, n, batch = 0x1234_5678_9ABC, 98000, 256
    step = torch.tensor([37], dtype=torch.int32, device="cuda")
    idx = torch.empty(batch, dtype=torch.int64, device="cuda")
    svk.svk_cnn_draw_batch(seed, step, n, idx)
    want = [((_splitmix64(seed + 37 * batch + i) >> 32) * n) >> 32 for i in range(batch)]
    assert idx.cpu().tolist() == want
    # the counter advances with the step: another step, another batch
    step.fill_(38)
    idx2 = svk.svk_cnn_draw_batch(seed, step, n, torch.empty_like(idx))
    assert not torch.equal(idx, idx2)
    # uniform over [0, n): 100 000 draws in 10 bins, chi-square with 9 degrees of freedom
    big = torch.empty(100000, dtype=torch.int64, device="cuda")
    step.fill_(0)
    svk.svk_cnn_draw_batch(7, step, 10, big)
    counts = np.bincount(big.cpu().numpy(), minlength=10)
    assert counts.min() >= 0 and big.min() >= 0 and big.max() < 10
    chi2 = (((counts - 10000.0) ** 2) / 10000.0).sum()
    assert chi2 < 27.9  # p = 0.001 for 9 degrees of freedom


def test_gather_rows_and_step_end():
    g = starfield.rng(204)
    src = torch.from_numpy(g.standard_normal((500, 2, 8, 8)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(g.standard_normal((500, 49)).astype(np.float32)).cuda()
    idx = torch.from_numpy(g.integers(0, 500, 77)).cuda()
    out = torch.empty((77, 2, 8, 8), device="cuda")
    outt = torch.empty((77, 49), device="cuda")
    svk.svk_gather_rows(src, idx, out)
    svk.svk_gather_rows(tgt, idx, outt)
    assert torch.equal(out, src[idx]) and torch.equal(outt, tgt[idx])
    step = torch.tensor([5], dtype=torch.int32, device="cuda")
    hist = torch.zeros(4, device="cuda")
    for k in range(6):
        svk.svk_cnn_step_end(torch.tensor([float(k)], device="cuda"), step, hist)
    assert int(step.item()) == 11
    # steps 5..10 wrote slots 1, 2, 3, 0, 1, 2
    assert hist.cpu().tolist() == [3.0, 4.0, 5.0, 2.0]
