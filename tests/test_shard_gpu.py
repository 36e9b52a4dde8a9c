"""The library calls behind the multi-GPU split of one frame, on one GPU: bands of output
rows from buffers that hold only the rows a band reads (svk_difference_rows), and the fit
split into moments of stamp subsets plus one solve (svk_fit_moments, svk_fit_solve).

The ranks of a split run one after another in this process (nothing waits on another
rank).  Rows outside what a band buffer should hold are NaN, so a read beyond them would
show in the result; band rows must equal the whole-frame call bit for bit (the bands are
aligned to the kernel's row block, so every pixel is summed in the same order).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1209_5823_gb300 as svk
import starfield
from _helpers import coeffs, star_pair
from paper_1209_5823_gb300 import shard

pytestmark = pytest.mark.gpu

PAD = 8  # poisoned rows around every band buffer

CASES = [
    (svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3),
    (svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3),
    (svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32),
    (svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3),
    (svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32),
]


def _poisoned(rows, W, pitch):
    """A [rows][W] view (row pitch `pitch`) inside a NaN buffer with PAD rows on each side."""
    buf = torch.full((rows + 2 * PAD, pitch), float("nan"), dtype=torch.float32, device="cuda")
    return buf, buf[PAD:PAD + rows, :W]


@pytest.mark.parametrize("method,prec", CASES)
@pytest.mark.parametrize("pitch_extra", [0, 37])
def test_bands_from_band_buffers_equal_whole_frame(method, prec, pitch_extra):
    W, H, L, d = 1000, 777, 19, 2
    R, I = star_pair(W, H, 800, 91)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    c = torch.from_numpy(coeffs(49, d, 92)).cuda()
    Rt, It = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda()
    full = svk.svk_difference(Rt, It, B, c, d, method=method, precision=prec)
    gran = svk.svk_band_rows(method, prec, 49, L, d)
    assert gran > 0
    h = L // 2
    for world in (2, 3):
        got = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        for band in shard.row_bands(H, gran, world):
            if band.y1 <= band.y0:
                continue
            r0, r1 = shard.held_rows(band, h, H)
            Rbuf, Rb = _poisoned(r1 - r0, W, W + pitch_extra)
            Rb.copy_(Rt[r0:r1])
            Ibuf, Ib = _poisoned(band.y1 - band.y0, W, W + pitch_extra)
            Ib.copy_(It[band.y0:band.y1])
            Dbuf, Db = _poisoned(band.y1 - band.y0, W, W + pitch_extra)
            svk.svk_difference_rows(Rb, Ib, B, c, d, W, H, band.y0, band.y1, r0, method=method, precision=prec,
                                    out=Db)
            got[band.y0:band.y1] = Db
            # nothing written outside the band's rows and columns
            Dh = Dbuf.cpu().numpy()
            assert np.isnan(Dh[:PAD]).all() and np.isnan(Dh[PAD + band.y1 - band.y0:]).all()
            assert np.isnan(Dh[:, W:]).all()
        assert torch.equal(got, full), (method, prec, world)


def test_band_of_a_plain_convolution_and_host_frames():
    # I = None gives rows of R (x) K; shard.difference_band takes pinned host frames
    W, H, L, d = 640, 512, 15, 1
    R, I = star_pair(W, H, 300, 93)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    c = torch.from_numpy(coeffs(49, d, 94)).cuda()
    Rt, It = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda()
    conv = svk.svk_convolve(Rt, B, c, d, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    gran = svk.svk_band_rows(svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3, 49, L, d)
    band = shard.row_bands(H, gran, 2)[1]
    r0, r1 = shard.held_rows(band, L // 2, H)
    part = svk.svk_difference_rows(Rt[r0:r1].contiguous(), None, B, c, d, W, H, band.y0, band.y1, r0)
    assert torch.equal(part, conv[band.y0:band.y1])
    full = svk.svk_difference(Rt, It, B, c, d, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    Rh, Ih = torch.from_numpy(R).pin_memory(), torch.from_numpy(I).pin_memory()
    got = torch.empty_like(full)
    for rank in range(3):
        Db, bd = shard.difference_band(Rh, Ih, B, c, d, svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3, rank=rank, world=3)
        got[bd.y0:bd.y1] = Db
    assert torch.equal(got, full)


def test_band_argument_checks():
    W, H, L, d = 256, 200, 11, 1
    R, I = star_pair(W, H, 50, 95)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    c = torch.from_numpy(coeffs(49, d, 96)).cuda()
    Rt, It = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda()
    gran = svk.svk_band_rows(svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32, 49, L, d)
    assert gran == 12
    # a band start off the row block, and a held range short of the halo
    with pytest.raises(svk.SvkError) as e:
        svk.svk_difference_rows(Rt, It[5:29], B, c, d, W, H, 5, 29, 0, method=svk.SVK_METHOD_DIRECT,
                                precision=svk.SVK_PREC_FP32)
    assert e.value.status == svk.SVK_ERR_ARG
    with pytest.raises(svk.SvkError) as e:
        svk.svk_difference_rows(Rt[24:60].contiguous(), It[24:48], B, c, d, W, H, 24, 48, 24,
                                method=svk.SVK_METHOD_DIRECT, precision=svk.SVK_PREC_FP32)
    assert e.value.status == svk.SVK_ERR_ARG
    assert svk.svk_band_rows(svk.SVK_METHOD_DIRECT, svk.SVK_PREC_BF16X3, 49, L, d) == 0


def _fit_setup(W, H, L, S, d, n, seed):
    R, _ = star_pair(W, H, W * H // 100, seed)
    B = oracle.gauss_basis(L).astype(np.float32)
    c = starfield.planted_coeffs(B.shape[0], d, starfield.rng(seed + 1))
    g = starfield.rng(seed + 2)
    xy = np.stack([g.integers(S, W - S, n), g.integers(0, H, n)], 1).astype(np.int32)  # some cross the edges
    hs = S // 2
    off = np.arange(-hs, hs + 1)
    px = np.clip((xy[:, 0][:, None, None] + off[None, None, :]).repeat(S, axis=1).ravel(), 0, W - 1).astype(np.int32)
    py = np.clip((xy[:, 1][:, None, None] + off[None, :, None]).repeat(S, axis=2).ravel(), 0, H - 1).astype(np.int32)
    m = oracle.convolve_points(R.astype(np.float64), B.astype(np.float64), c, d, px, py)
    I = R.copy()
    I[py, px] = (m + 7.0 + g.normal(0.0, 30.0, m.shape)).astype(np.float32)
    return R, I, B, xy, px, py


def test_fit_moments_summed_over_bands_equal_the_whole_fit():
    W, H, L, S, d, bd = 1024, 1024, 25, 41, 3, 0
    R, I, B, xy, px, py = _fit_setup(W, H, L, S, d, 90, 97)
    Rt, It, Bt = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), torch.from_numpy(B).cuda()
    st = torch.from_numpy(xy).cuda()
    N = B.shape[0]
    co_full, chi2_full, info_full = svk.svk_fit_coeffs(Rt, It, st, S, Bt, d, bg_degree=bd, sync=True)
    whole = svk.svk_fit_moments(Rt, It, st, S, Bt, d, bd)
    co_w, chi2_w, info_w = svk.svk_fit_solve(whole, N, d, bd, sync=True)
    assert int(info_w.item()) == -1
    for world in (2, 3):
        total = torch.zeros_like(whole)
        for band in shard.row_bands(H, 1, world):
            own = shard.stamps_of(xy, band)
            r0, r1 = shard.held_rows(band, shard.fit_halo(S, L), H)
            _, Rb = _poisoned(r1 - r0, W, W)
            Rb.copy_(Rt[r0:r1])
            _, Ib = _poisoned(r1 - r0, W, W)
            Ib.copy_(It[r0:r1])
            stb = torch.from_numpy(xy[own]).cuda() if len(own) else None
            # accumulate into one array, as a rank would before the all-reduce
            svk.svk_fit_moments(Rb, Ib, stb, S, Bt, d, bd, W=W, H=H, row_begin=r0, moments=total, accumulate=True)
        a, b = total.cpu().numpy(), whole.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(b).max())
        co, chi2, info = svk.svk_fit_solve(total, N, d, bd, sync=True)
        assert int(info.item()) == -1
        # the fitted model at every stamp pixel against the whole-frame fit's (oracle evaluation)
        T = oracle.n_terms(d)

        def model(cv):
            cv = np.asarray(cv, dtype=np.float64)
            return oracle.convolve_points(R.astype(np.float64), B.astype(np.float64), cv[:N * T].reshape(N, T), d,
                                          px, py) + cv[N * T]

        dm = model(co.cpu().numpy()) - model(co_full.cpu().numpy())
        assert np.abs(dm).max() <= 1e-3 * 30.0
        # chi^2 from the moments against the direct pass over the pixels
        assert abs(float(chi2.item()) - float(chi2_full.item())) <= 1e-6 * float(chi2_full.item())
    assert abs(float(chi2_w.item()) - float(chi2_full.item())) <= 1e-6 * float(chi2_full.item())


def test_fit_moments_edge_cases():
    W, H, L, S, d = 256, 256, 11, 21, 1
    R, I, B, xy, _, _ = _fit_setup(W, H, L, S, d, 12, 98)
    Rt, It, Bt = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), torch.from_numpy(B).cuda()
    n = svk.svk_fit_moments_count(49, d, -1)
    assert n == 51 * 51 * oracle.n_terms(2 * d)
    # no stamps: zero moments, and accumulating nothing leaves them unchanged
    z = svk.svk_fit_moments(Rt, It, None, S, Bt, d, -1)
    assert z.numel() == n and torch.count_nonzero(z) == 0
    m = svk.svk_fit_moments(Rt, It, torch.from_numpy(xy).cuda(), S, Bt, d, -1)
    m2 = m.clone()
    svk.svk_fit_moments(Rt, It, None, S, Bt, d, -1, moments=m2, accumulate=True)
    assert torch.equal(m, m2)
    # one fit through the host-memory sharding path on a single process equals the device fit
    Rh, Ih = torch.from_numpy(R), torch.from_numpy(I)
    co, chi2, info = shard.fit_coeffs(Rh, Ih, xy, S, Bt, d, -1, rank=0, world=1, sync=True)
    co2, chi22, info2 = svk.svk_fit_solve(m, 49, d, -1, sync=True)
    # the same moments up to the order of the FP64 atomic sums: the same optimum
    assert int(info.item()) == -1 and int(info2.item()) == -1
    assert abs(float(chi2.item()) - float(chi22.item())) <= 1e-8 * float(chi22.item())
