"""Parity of the device least-squares fit (FP32 C_k, FP64 normal equations, FP64 Cholesky)
with the FP64 oracle fit, on seeded star fields with planted coefficients."""
import numpy as np
import pytest
import torch

import oracle
import paper_1209_5823_gb300 as svk
import starfield
from _helpers import star_pair

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _stamps(W, H, n, margin, seed):
    g = starfield.rng(seed)
    return np.stack([g.integers(margin, W - margin, n), g.integers(margin, H - margin, n)], axis=1).astype(np.int32)


def _setup(W, H, L, S, d, n_stamps, sigma, deg, seed, noise=0.0, bg=None):
    R, _ = star_pair(W, H, max(10, W * H // 80), seed)
    B = oracle.gauss_basis(L, sigma=sigma, deg=deg).astype(np.float32)
    N = B.shape[0]
    c = starfield.planted_coeffs(N, d, starfield.rng(seed + 1), const_sd=0.1, spatial_sd=0.05)
    I = oracle.convolve(R.astype(np.float64), B.astype(np.float64), c, d)
    if bg is not None:
        X, Y = np.meshgrid(np.linspace(-1, 1, W), np.linspace(-1, 1, H))
        I = I + bg[0] + bg[1] * Y + bg[2] * X
    if noise:
        I = I + starfield.rng(seed + 2).normal(0, noise, I.shape)
    I = I.astype(np.float32)
    st = _stamps(W, H, n_stamps, (S - 1) // 2 + 2, seed + 3)
    return R, I, B, c, st


def test_fit_recovers_planted_and_matches_oracle():
    W, H, L, S, d = 96, 80, 7, 11, 1
    R, I, B, c, st = _setup(W, H, L, S, d, 16, (0.9, 1.8), (1, 0), 40)
    ref = oracle.fit(R.astype(np.float64), I.astype(np.float64), st, S, B.astype(np.float64), d)
    co, chi2, info = svk.svk_fit_coeffs(_dev(R), _dev(I), _dev(st), S, _dev(B), d, sync=True)
    co = co.cpu().numpy()
    assert int(info.item()) == -1 and ref["status"] == 0
    np.testing.assert_allclose(co, ref["coeffs"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(co, c.reshape(-1), rtol=0, atol=2e-5)


@pytest.mark.parametrize("d,bd", [(0, 2), (1, 3)])
def test_fit_background_above_kernel_degree(d, bd):
    # a background polynomial of higher degree than the kernel's: the monomials of both
    # (degree max(d, bd)) and their moments (degree 2 max(d, bd)) index past the kernel terms'
    W, H, L, S, sig = 128, 96, 9, 13, 10.0
    R, I, B, c, st = _setup(W, H, L, S, d, 30, (0.8, 1.6), (2, 1), 70 + bd, noise=sig, bg=(12.0, -3.0, 5.0))
    w = np.full((H, W), 1.0 / sig ** 2, np.float32)  # A is then the inverse covariance
    ref = oracle.fit(R.astype(np.float64), I.astype(np.float64), st, S, B.astype(np.float64), d, bg_degree=bd,
                     weight=w.astype(np.float64))
    co, chi2, info = svk.svk_fit_coeffs(_dev(R), _dev(I), _dev(st), S, _dev(B), d, bg_degree=bd, weight=_dev(w),
                                        sync=True)
    assert int(info.item()) == -1 and ref["status"] == 0
    assert abs(float(chi2.item()) - ref["chi2"]) <= 1e-4 * ref["chi2"]
    # coefficients agree to a small fraction of their statistical uncertainty
    cov = np.linalg.inv(ref["A"])
    z = (co.cpu().numpy() - ref["coeffs"]) / np.sqrt(np.diag(cov))
    assert np.abs(z).max() < 1e-2


def test_fit_background_weights_noise_chi2():
    W, H, L, S, d, bd = 128, 96, 9, 13, 2, 1
    sig = 30.0
    R, I, B, c, st = _setup(W, H, L, S, d, 24, (0.8, 1.6), (2, 1), 50, noise=sig, bg=(12.0, -3.0, 5.0))
    w = np.full((H, W), 1.0 / sig ** 2, np.float32)
    ref = oracle.fit(R.astype(np.float64), I.astype(np.float64), st, S, B.astype(np.float64), d, bg_degree=bd,
                     weight=w.astype(np.float64))
    co, chi2, info = svk.svk_fit_coeffs(_dev(R), _dev(I), _dev(st), S, _dev(B), d, bg_degree=bd, weight=_dev(w),
                                        sync=True)
    assert int(info.item()) == -1
    g = float(chi2.item())
    assert abs(g - ref["chi2"]) <= 1e-4 * ref["chi2"]
    # coefficients agree to a small fraction of their statistical uncertainty
    cov = np.linalg.inv(ref["A"])
    z = (co.cpu().numpy() - ref["coeffs"]) / np.sqrt(np.diag(cov))
    assert np.abs(z).max() < 1e-2


def test_fit_full_49_stamp_basis_d3():
    # the 49-stamp Gaussian basis with cubic spatial variation (490 unknowns + background)
    W, H, L, S, d, bd = 256, 224, 11, 21, 3, 0
    R, I, B, c, st = _setup(W, H, L, S, d, 60, (0.7, 1.5, 2.5), (6, 4, 2), 60, noise=5.0, bg=(7.0, 0.0, 0.0))
    ref = oracle.fit(R.astype(np.float64), I.astype(np.float64), st, S, B.astype(np.float64), d, bg_degree=bd)
    co, chi2, info = svk.svk_fit_coeffs(_dev(R), _dev(I), _dev(st), S, _dev(B), d, bg_degree=bd, sync=False)
    torch.cuda.synchronize()
    # seed 60 gives a positive definite oracle matrix (checked on the CPU): no skip path
    assert ref["status"] == 0
    assert int(info.item()) == -1
    # the D residual is what the fit is for; ill-conditioned directions may differ
    assert abs(float(chi2.item()) - ref["chi2"]) <= 1e-3 * ref["chi2"]
    # the fitted model at every stamp pixel (sum_k a_k C_k + bg), device coefficients
    # against the oracle's, both evaluated by the oracle
    N, T = B.shape[0], oracle.n_terms(d)
    hs = (S - 1) // 2
    off = np.arange(-hs, hs + 1)
    px = (st[:, 0][:, None, None] + off[None, None, :]).repeat(S, axis=1).ravel().astype(np.int32)
    py = (st[:, 1][:, None, None] + off[None, :, None]).repeat(S, axis=2).ravel().astype(np.int32)

    def model(cv):
        cv = np.asarray(cv, dtype=np.float64)
        return oracle.convolve_points(R.astype(np.float64), B.astype(np.float64), cv[:N * T].reshape(N, T), d,
                                      px, py) + cv[N * T]

    dm = model(co.cpu().numpy()) - model(ref["coeffs"])
    assert np.sqrt(np.mean(dm * dm)) <= 1e-3 * 5.0 and np.abs(dm).max() <= 2e-2 * 5.0


def test_fit_reports_not_positive_definite():
    W, H, L, S = 64, 64, 5, 7
    R, _ = star_pair(W, H, 30, 70)
    B = oracle.gauss_basis(L, sigma=(1.0,), deg=(0,), normalize=oracle.NORM_NONE).astype(np.float32)
    B2 = np.concatenate([B, 0.0 * B], axis=0)  # an all-zero stamp: its pivot is exactly 0
    st = _stamps(W, H, 6, 5, 71)
    co, chi2, info = svk.svk_fit_coeffs(_dev(R), _dev(R), _dev(st), S, _dev(B2), 0)
    torch.cuda.synchronize()
    assert int(info.item()) >= 0
    assert np.all(co.cpu().numpy() == 0.0)
    with pytest.raises(svk.SvkError) as e:
        svk.svk_fit_coeffs(_dev(R), _dev(R), _dev(st), S, _dev(B2), 0, sync=True)
    assert e.value.status == svk.SVK_ERR_NOT_SPD
