"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle through a route that does not reuse its own formula:
library convolutions (scipy FFT / direct), closed forms of delta bases, impulse
responses, flux conservation, the cost-model numbers printed in Sec. 3, numpy's
Cholesky and planted-coefficient recovery.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

import oracle
import starfield

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _star_R(W, H, n, seed, sky=1000.0):
    g = starfield.rng(seed)
    cat = starfield.star_catalog(W, H, n, g)
    return starfield.add_noise(starfield.render(cat, W, H, sky=sky), 30.0, g)


def _coords(W, H):
    # normalised coordinates built from linspace, not from the oracle's formula
    xt = np.linspace(-1.0, 1.0, W) if W > 1 else np.zeros(1)
    yt = np.linspace(-1.0, 1.0, H) if H > 1 else np.zeros(1)
    return np.meshgrid(xt, yt)


def _poly_field(c_row, degree, W, H):
    """sum_t c_t xt^i yt^j with t over i outer, j inner (Eq. 3 order for d = 2)."""
    X, Y = _coords(W, H)
    out = np.zeros((H, W))
    t = 0
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            out += c_row[t] * X ** i * Y ** j
            t += 1
    return out


# ---------------------------------------------------------------- cost models (Sec. 3)
def _golden_flops():
    vals = {}
    with open(os.path.join(GOLDEN, "flop_models.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, digits = line.split()
            vals[name] = (float(value), digits)
    return vals


def _agrees(x, printed, digits):
    if digits == "exact":
        return x == printed
    d = int(digits)
    return float(f"{x:.{d}g}") == printed


def test_flop_models_match_printed_values():
    g = _golden_flops()
    tile = 4846 * 4868
    dfb = oracle.flops_dfb_per_pixel(7)
    gfb = oracle.flops_gfb_per_pixel(3, 7)
    assert _agrees(dfb, *g["dfb_flop_per_pixel_L7"])
    assert _agrees(dfb * tile / 1e9, *g["dfb_gflop_per_tile_L7"])
    assert _agrees(dfb * tile * 60 / 1e12, *g["dfb_tflop_per_image_L7"])
    assert _agrees(gfb, *g["gfb_flop_per_pixel_N3_L7"])
    assert _agrees(gfb * tile / 1e9, *g["gfb_gflop_per_tile_N3_L7"])
    assert _agrees(gfb * tile * 60 / 1e9, *g["gfb_gflop_per_image_N3_L7"])


# ---------------------------------------------------------------- coordinates / monomials
def test_norm_coord_and_monomial_order():
    assert oracle.norm_coord(0, 5) == -1.0 and oracle.norm_coord(4, 5) == 1.0
    assert oracle.norm_coord(2, 5) == 0.0 and oracle.norm_coord(0, 1) == 0.0
    x, y = 0.3, -0.7
    # Eq. 3: a00 + a01 y + a02 y^2 + a11 xy + a10 x + a20 x^2  (our order: 1, y, y^2, x, xy, x^2)
    np.testing.assert_allclose(oracle.monomials(x, y, 2), [1, y, y * y, x, x * y, x * x], rtol=0, atol=0)
    assert [oracle.n_terms(d) for d in range(4)] == [1, 3, 6, 10]


# ---------------------------------------------------------------- basis stamps
def test_gauss_basis_count_and_closed_form_values():
    B = oracle.gauss_basis(11)
    assert B.shape == (49, 11, 11)  # 28 + 15 + 6
    # raw stamps: sigma = 1, degree 1 -> (p, q) = (0,0), (0,1), (1,0)
    R = oracle.gauss_basis(3, sigma=(1.0,), deg=(1,), normalize=oracle.NORM_NONE)
    e = math.exp(-0.5)
    # index [v + h][u + h]; (u, v) = (1, 0) -> [1][2]; (u, v) = (0, 1) -> [2][1]
    assert R[0][1][1] == 1.0 and abs(R[0][1][2] - e) < 1e-16 and abs(R[0][0][0] - math.exp(-1.0)) < 1e-16
    assert R[1][1][2] == 0.0 and abs(R[1][2][1] - e) < 1e-16 and abs(R[1][0][1] + e) < 1e-16  # v^1
    assert R[2][2][1] == 0.0 and abs(R[2][1][2] - e) < 1e-16 and abs(R[2][1][0] + e) < 1e-16  # u^1


def test_gauss_basis_alard_normalisation():
    B = oracle.gauss_basis(19)
    sums = B.reshape(49, -1).sum(axis=1)
    assert abs(sums[0] - 1.0) < 1e-14
    assert np.max(np.abs(sums[1:])) < 1e-13
    norms = np.sqrt((B[1:].reshape(48, -1) ** 2).sum(axis=1))
    np.testing.assert_allclose(norms, 1.0, rtol=1e-13)


def test_delta_basis():
    D = oracle.delta_basis(5)
    assert np.array_equal(D.reshape(25, 25), np.eye(25))
    A = oracle.delta_basis(5, oracle.NORM_ALARD)
    s = A.reshape(25, -1).sum(axis=1)
    assert s[12] == 1.0 and np.all(np.delete(s, 12) == 0.0)


# ---------------------------------------------------------------- convolution special cases
def test_identity_delta_centre():
    R = _star_R(37, 29, 20, 1)
    B = oracle.delta_basis(5)
    c = np.zeros((25, 1))
    c[12, 0] = 1.0
    out = oracle.convolve(R, B, c, 0)
    assert np.array_equal(out, R)


def test_delta_shift_pins_convolution_flip():
    R = _star_R(31, 23, 15, 2)
    L, h = 5, 2
    B = oracle.delta_basis(L)
    for (u0, v0) in [(1, 0), (0, 2), (-2, 1)]:
        c = np.zeros((L * L, 1))
        c[(v0 + h) * L + (u0 + h), 0] = 1.0
        out = oracle.convolve(R, B, c, 0)
        # true convolution: out(x, y) = R(x - u0, y - v0), zero outside
        exp = np.zeros_like(R)
        H, W = R.shape
        ys, xs = np.mgrid[0:H, 0:W]
        src_x, src_y = xs - u0, ys - v0
        ok = (src_x >= 0) & (src_x < W) & (src_y >= 0) & (src_y < H)
        exp[ok] = R[src_y[ok], src_x[ok]]
        assert np.array_equal(out, exp)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_spatially_varying_delta_closed_form(degree):
    W, H = 41, 26
    R = _star_R(W, H, 25, 3)
    L = 3
    B = oracle.delta_basis(L)
    g = starfield.rng(11)
    T = oracle.n_terms(degree)
    c = np.zeros((L * L, T))
    c[4] = g.normal(0, 0.3, T)
    out = oracle.convolve(R, B, c, degree)
    exp = _poly_field(c[4], degree, W, H) * R
    np.testing.assert_allclose(out, exp, rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize("L", [1, 5, 11])
def test_constant_coeffs_match_fft_and_direct_library(L):
    W, H = 47, 38  # ragged, not square
    R = _star_R(W, H, 30, 4)
    B = oracle.gauss_basis(L) if L > 1 else oracle.delta_basis(1)
    N = B.shape[0]
    c = starfield.planted_coeffs(N, 0, starfield.rng(5))
    out = oracle.convolve(R, B, c, 0)
    K = np.tensordot(c[:, 0], B, axes=1)
    fft = scipy.signal.fftconvolve(R, K, mode="same")
    direct = scipy.ndimage.convolve(R, K, mode="constant", cval=0.0)
    scale = np.abs(out).max()
    assert np.abs(out - fft).max() <= 1e-10 * scale
    assert np.abs(out - direct).max() <= 1e-12 * scale


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_spatially_varying_equals_sum_of_library_convolutions(degree):
    """R (x) K_{x,y} = sum_k a_k(x,y) (R (x) B_k)(x,y): linearity of Eq. 2, each R (x) B_k by scipy."""
    W, H = 40, 33
    R = _star_R(W, H, 25, 6)
    L = 7
    B = oracle.gauss_basis(L)
    N = B.shape[0]
    c = starfield.planted_coeffs(N, degree, starfield.rng(7), const_sd=0.3, spatial_sd=0.2)
    out = oracle.convolve(R, B, c, degree)
    exp = np.zeros((H, W))
    for k in range(N):
        exp += _poly_field(c[k], degree, W, H) * scipy.signal.convolve2d(R, B[k], mode="same",
                                                                       boundary="fill", fillvalue=0.0)
    assert np.abs(out - exp).max() <= 1e-11 * np.abs(exp).max()


def test_impulse_response_is_kernel_at_output_pixel():
    W, H, L, h = 23, 21, 7, 3
    x0, y0 = 11, 9
    R = np.zeros((H, W))
    R[y0, x0] = 1.0
    B = oracle.gauss_basis(L)
    N = B.shape[0]
    c = starfield.planted_coeffs(N, 2, starfield.rng(8), const_sd=0.3, spatial_sd=0.5, scale_sd=0.5)
    out = oracle.convolve(R, B, c, 2)
    for y in range(y0 - h, y0 + h + 1):
        for x in range(x0 - h, x0 + h + 1):
            a = np.array([_poly_field(c[k], 2, W, H)[y, x] for k in range(N)])
            K = np.tensordot(a, B, axes=1)  # the kernel of the OUTPUT pixel
            assert abs(out[y, x] - K[(y - y0) + h, (x - x0) + h]) <= 1e-12
    # zero outside the kernel footprint
    mask = np.ones_like(out, dtype=bool)
    mask[y0 - h:y0 + h + 1, x0 - h:x0 + h + 1] = False
    assert np.all(out[mask] == 0.0)


def test_flux_conservation_alard():
    W, H, L = 64, 48, 11
    R = np.zeros((H, W))
    g = starfield.rng(9)
    for _ in range(12):  # compact sources at least h + 3 px from the edges
        x, y = g.integers(9, W - 9), g.integers(9, H - 9)
        R[y - 1:y + 2, x - 1:x + 2] += g.uniform(1e3, 1e5)
    B = oracle.gauss_basis(L)
    c = starfield.planted_coeffs(B.shape[0], 0, g)
    out = oracle.convolve(R, B, c, 0)
    assert abs(out.sum() - R.sum()) <= 1e-12 * R.sum()


def test_linearity():
    W, H, L = 30, 22, 5
    R1, R2 = _star_R(W, H, 10, 10), _star_R(W, H, 10, 11)
    B = oracle.gauss_basis(L)
    N = B.shape[0]
    c1 = starfield.planted_coeffs(N, 2, starfield.rng(12))
    c2 = starfield.planted_coeffs(N, 2, starfield.rng(13))
    f = lambda R, c: oracle.convolve(R, B, c, 2)
    s = np.abs(f(R1, c1)).max()
    assert np.abs(f(R1 + 2.5 * R2, c1) - f(R1, c1) - 2.5 * f(R2, c1)).max() <= 1e-12 * s
    assert np.abs(f(R1, c1 - 0.5 * c2) - f(R1, c1) + 0.5 * f(R1, c2)).max() <= 1e-12 * s


def test_difference_rows_points_consistent():
    W, H, L = 33, 27, 7
    R = _star_R(W, H, 15, 14)
    I = _star_R(W, H, 15, 15)
    B = oracle.gauss_basis(L)
    c = starfield.planted_coeffs(B.shape[0], 1, starfield.rng(16))
    full = oracle.convolve(R, B, c, 1)
    assert np.array_equal(oracle.difference(R, I, B, c, 1), full - I)
    assert np.array_equal(oracle.convolve(R, B, c, 1, rows=(5, 19)), full[5:19])
    px = np.array([0, 32, 5, 17, 31])
    py = np.array([0, 26, 13, 1, 20])
    assert np.array_equal(oracle.convolve_points(R, B, c, 1, px, py), full[py, px])


def test_degenerate_sizes():
    R = np.array([[3.0]])
    B = oracle.gauss_basis(5)
    c = starfield.planted_coeffs(B.shape[0], 2, starfield.rng(17))
    out = oracle.convolve(R, B, c, 2)
    # 1x1 frame: only the centre tap sees R; coordinates are 0 so only t = 0 terms act
    assert abs(out[0, 0] - 3.0 * np.dot(c[:, 0], B[:, 2, 2])) <= 1e-14
    row = _star_R(17, 1, 3, 18)
    out = oracle.convolve(row, B, c, 2)
    assert out.shape == (1, 17)


# ---------------------------------------------------------------- Cholesky and the fit
def test_cholesky_matches_numpy():
    g = starfield.rng(19)
    X = g.normal(size=(40, 25))
    A = X.T @ X + 0.1 * np.eye(25)
    G, piv = oracle.cholesky(A)
    assert piv == -1
    np.testing.assert_allclose(G, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    b = g.normal(size=25)
    np.testing.assert_allclose(oracle.cholesky_solve(G, b), np.linalg.solve(A, b), rtol=1e-10)


def test_cholesky_reports_first_bad_pivot():
    A = np.diag([2.0, 1.0, -1.0, 4.0])
    _, piv = oracle.cholesky(A)
    assert piv == 2
    A = np.array([[1.0, 2.0], [2.0, 4.0]])  # singular: second pivot is exactly 0
    assert oracle.cholesky(A)[1] == 1


def _stamps(W, H, n, margin, g):
    return np.stack([g.integers(margin, W - margin, n), g.integers(margin, H - margin, n)], axis=1)


def test_normal_equations_match_design_matrix_from_library_convolutions():
    W, H, L, S, d, bd = 44, 36, 5, 7, 2, 1
    R = _star_R(W, H, 25, 20)
    I = _star_R(W, H, 25, 21)
    B = oracle.gauss_basis(L, sigma=(0.8, 1.6), deg=(2, 1))
    N = B.shape[0]
    st = _stamps(W, H, 6, 4, starfield.rng(22))
    A, b = oracle.normal_equations(R, I, st, S, B, d, bg_degree=bd)
    Ck = [scipy.signal.convolve2d(R, B[k], mode="same") for k in range(N)]
    T = oracle.n_terms(d)
    rows, rhs = [], []
    X, Y = _coords(W, H)
    for (cx, cy) in st:
        for y in range(cy - 3, cy + 4):
            for x in range(cx - 3, cx + 4):
                mon = []
                for i in range(d + 1):
                    for j in range(d + 1 - i):
                        mon.append(X[y, x] ** i * Y[y, x] ** j)
                bg = []
                for i in range(bd + 1):
                    for j in range(bd + 1 - i):
                        bg.append(X[y, x] ** i * Y[y, x] ** j)
                rows.append([mon[t] * Ck[k][y, x] for k in range(N) for t in range(T)] + bg)
                rhs.append(I[y, x])
    V = np.array(rows)
    np.testing.assert_allclose(A, V.T @ V, rtol=1e-10, atol=1e-9 * np.abs(A).max())
    np.testing.assert_allclose(b, V.T @ np.array(rhs), rtol=1e-10, atol=1e-9 * np.abs(b).max())


def test_fit_recovers_planted_coefficients_noise_free():
    W, H, L, S, d = 48, 40, 7, 9, 1
    R = _star_R(W, H, 40, 23)
    B = oracle.gauss_basis(L, sigma=(0.9, 1.8), deg=(1, 0))
    N = B.shape[0]
    c = starfield.planted_coeffs(N, d, starfield.rng(24), const_sd=0.1, spatial_sd=0.05)
    I = oracle.convolve(R, B, c, d)
    st = _stamps(W, H, 12, 5, starfield.rng(25))
    res = oracle.fit(R, I, st, S, B, d)
    assert res["status"] == 0 and res["info"] == -1
    np.testing.assert_allclose(res["coeffs"], c.reshape(-1), rtol=0, atol=1e-8)
    assert res["chi2"] <= 1e-12 * (I ** 2).sum()


def test_fit_with_background_and_noise_chi2_per_dof():
    W, H, L, S, d, bd = 64, 56, 7, 11, 1, 1
    g = starfield.rng(26)
    R = _star_R(W, H, 60, 27)
    B = oracle.gauss_basis(L, sigma=(0.9, 1.8), deg=(2, 0))
    N = B.shape[0]
    c = starfield.planted_coeffs(N, d, starfield.rng(28), const_sd=0.1, spatial_sd=0.05)
    bg = np.array([12.0, -3.0, 5.0])  # 1, y, x
    X, Y = _coords(W, H)
    sigma = 30.0
    I = oracle.convolve(R, B, c, d) + bg[0] + bg[1] * Y + bg[2] * X + g.normal(0, sigma, (H, W))
    st = _stamps(W, H, 20, 6, starfield.rng(29))
    w = np.full((H, W), 1.0 / sigma ** 2)
    res = oracle.fit(R, I, st, S, B, d, bg_degree=bd, weight=w)
    assert res["status"] == 0
    n_px = len(st) * S * S
    dof = n_px - (N * oracle.n_terms(d) + 3)
    # chi^2 of Gaussian noise with unit weight per pixel: mean dof, sd sqrt(2 dof)
    assert abs(res["chi2"] - dof) < 6 * math.sqrt(2 * dof)
    # the fitted model explains the planted signal to the noise level
    assert np.all(np.abs(res["coeffs"][-3:] - bg) < 10.0)


def test_fit_reports_non_spd():
    W, H, L, S = 30, 30, 5, 7
    R = _star_R(W, H, 10, 30)
    B = oracle.gauss_basis(L, sigma=(1.0,), deg=(0,), normalize=oracle.NORM_NONE)
    B2 = np.concatenate([B, B], axis=0)  # duplicated stamp: exactly singular normal matrix
    st = _stamps(W, H, 3, 4, starfield.rng(31))
    res = oracle.fit(R, R, st, S, B2, 0)
    assert res["status"] == oracle.ERR_NOT_SPD and res["info"] == 1
