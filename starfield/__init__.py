"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the image-subtraction method itself: it draws star
catalogues, renders them with Gaussian point-spread functions, adds sky and noise, and
draws planted polynomial coefficients.  Convolving with the spatially-varying kernel
(Eq. 2) is the job of the oracle and of the CUDA library, never of this module.

Star-field model (stands in for the survey CCD frames the paper processes in Sec. 3
and Sec. 5; the real NEAT / Pan-STARRS images are not available):

* star centres uniform over the frame, FWHM uniform in [2, 4] px
  (sigma = FWHM / 2.3548), the PSF evaluated at pixel centres;
* fluxes log-uniform in [1e3, 1e5] counts;
* sky level 1000 counts, Gaussian read noise sigma = 30 counts;
* all draws from numpy ``Generator(Philox(seed))`` with seed 20121205 + config index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20121205
FWHM_TO_SIGMA = 1.0 / 2.3548200450309493


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator used everywhere in the repo (Philox4x64)."""
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclass
class Catalog:
    x: np.ndarray  # column centre (float, pixel units, pixel centres at integers)
    y: np.ndarray  # row centre
    sigma: np.ndarray  # Gaussian sigma in px
    flux: np.ndarray  # total counts


def star_catalog(W: int, H: int, n_stars: int, g: np.random.Generator,
                 fwhm=(2.0, 4.0), flux=(1e3, 1e5)) -> Catalog:
    x = g.uniform(0.0, W, n_stars)
    y = g.uniform(0.0, H, n_stars)
    fw = g.uniform(fwhm[0], fwhm[1], n_stars)
    lf = g.uniform(math.log(flux[0]), math.log(flux[1]), n_stars)
    return Catalog(x=x, y=y, sigma=fw * FWHM_TO_SIGMA, flux=np.exp(lf))


def render(cat: Catalog, W: int, H: int, sky: float = 1000.0, extra_sigma=None,
           flux_scale=None) -> np.ndarray:
    """Render a catalogue as circular Gaussians sampled at pixel centres (float64).

    ``extra_sigma(x, y)`` optionally broadens each star's PSF in quadrature and
    ``flux_scale(x, y)`` multiplies its flux; both describe a second epoch observed
    through different seeing, rendered directly from the star model.
    """
    img = np.full((H, W), float(sky), dtype=np.float64)
    if len(cat.x) == 0:
        return img
    sig = cat.sigma.copy()
    fl = cat.flux.copy()
    if extra_sigma is not None:
        sig = np.sqrt(sig ** 2 + np.asarray(extra_sigma(cat.x, cat.y)) ** 2)
    if flux_scale is not None:
        fl = fl * np.asarray(flux_scale(cat.x, cat.y))
    hw = int(math.ceil(5.0 * float(sig.max())))
    off = np.arange(-hw, hw + 1)
    # process in chunks to bound memory
    chunk = max(1, 4_000_000 // (len(off) ** 2))
    flat = img.reshape(-1)
    for s in range(0, len(cat.x), chunk):
        xs, ys = cat.x[s:s + chunk], cat.y[s:s + chunk]
        sg, fx = sig[s:s + chunk], fl[s:s + chunk]
        cx = np.floor(xs).astype(np.int64)
        cy = np.floor(ys).astype(np.int64)
        px = cx[:, None] + off[None, :]  # (n, w)
        py = cy[:, None] + off[None, :]
        gx = np.exp(-0.5 * ((px - xs[:, None]) / sg[:, None]) ** 2)
        gy = np.exp(-0.5 * ((py - ys[:, None]) / sg[:, None]) ** 2)
        amp = fx / (2.0 * math.pi * sg ** 2)
        val = amp[:, None, None] * gy[:, :, None] * gx[:, None, :]
        ok = (py[:, :, None] >= 0) & (py[:, :, None] < H) & (px[:, None, :] >= 0) & (px[:, None, :] < W)
        idx = py[:, :, None] * W + px[:, None, :]
        np.add.at(flat, idx[ok], val[ok])
    return img


def add_noise(img: np.ndarray, sigma: float, g: np.random.Generator) -> np.ndarray:
    return img + g.normal(0.0, sigma, img.shape)


def n_terms(degree: int) -> int:
    """Number of monomials x^i y^j with i + j <= degree (0 for degree < 0)."""
    return 0 if degree < 0 else (degree + 1) * (degree + 2) // 2


def planted_coeffs(N: int, degree: int, g: np.random.Generator, const_sd: float = 0.02,
                   spatial_sd: float = 0.01, scale_sd: float = 0.02) -> np.ndarray:
    """Planted polynomial coefficients c[k][t] (float64, shape N x T).

    c[0][0] = 1 (photometric scale of a unit-sum first basis), c[0][t>0] ~ N(0, scale_sd^2),
    c[k>0][0] ~ N(0, const_sd^2) and c[k>0][t>0] ~ N(0, spatial_sd^2), in normalised
    frame coordinates.
    """
    T = n_terms(degree)
    c = np.empty((N, T), dtype=np.float64)
    c[:, 0] = g.normal(0.0, const_sd, N)
    c[0, 0] = 1.0
    if T > 1:
        c[1:, 1:] = g.normal(0.0, spatial_sd, (N - 1, T - 1))
        c[0, 1:] = g.normal(0.0, scale_sd, T - 1)
    return c


# Alard-Lupton style Gaussian basis used by every config: 3 Gaussians of sigma 0.7 / 1.5 /
# 2.5 px times monomials of total degree <= 6 / 4 / 2, which gives 28 + 15 + 6 = 49 stamps.
GAUSS_SIGMA = (0.7, 1.5, 2.5)
GAUSS_DEG = (6, 4, 2)


@dataclass
class FrameSpec:
    name: str
    W: int  # columns
    H: int  # rows
    n_stars: int
    L: int
    degree: int
    seed: int
    extra: dict = field(default_factory=dict)


def _density_stars(W, H):
    # cfg1 density: ~20k stars on 2048 x 4096
    return int(round(20000 * (W * H) / (2048 * 4096)))


# the workloads by name: a 256^2 star field (L = 11, linear coefficients), the 2048-row x
# 4096-column CCD frame (L = 19, quadratic) and the 4096^2 frame (L = 25, cubic, with the
# fit's 500 stamps of 41 x 41)
WORKLOADS = {spec.name: spec for spec in (
    FrameSpec("starfield_256x256_L11_d1", 256, 256, 200, 11, 1, BASE_SEED + 0),
    FrameSpec("ccd_2048x4096_L19_d2", 4096, 2048, 20000, 19, 2, BASE_SEED + 1),
    FrameSpec("ccd_4096x4096_L25_d3", 4096, 4096, _density_stars(4096, 4096), 25, 3,
              BASE_SEED + 2, extra=dict(n_stamps=500, stamp_size=41)),
)}


def batch_specs(n_frames: int = 60, seed: int = BASE_SEED + 3, scale: float = 1.0):
    """The night-batch workload: a seeded mix of 2048^2, 2048x4096 and 4096^2 frames.

    One third of each size, seeded order; kernel size L in {15,17,...,31} and spatial degree
    d in {0..3} drawn per frame.  ``scale`` shrinks every side (for quick tests).
    """
    g = rng(seed)
    sizes = [(2048, 2048), (4096, 2048), (4096, 4096)]
    kinds = np.array([i % 3 for i in range(n_frames)])
    g.shuffle(kinds)
    Ls = g.choice(np.arange(15, 32, 2), n_frames)
    ds = g.integers(0, 4, n_frames)
    out = []
    for i in range(n_frames):
        W, H = sizes[kinds[i]]
        W = max(16, int(W * scale))
        H = max(16, int(H * scale))
        out.append(FrameSpec(f"night_{i:02d}_{W}x{H}_L{Ls[i]}_d{ds[i]}", W, H,
                             _density_stars(W, H), int(Ls[i]), int(ds[i]), seed * 100 + i))
    return out


def frame_pair(spec: FrameSpec, with_second_epoch: bool = True):
    """(R, I_seeing, catalog): R = star field + noise; I_seeing = the same field rendered
    through broader, position-dependent seeing, plus a different noise draw.

    ``I_seeing`` is a realistic second epoch for timing and for the fit; tests that need
    I = R (x) K + noise build it through the oracle instead.
    """
    g = rng(spec.seed)
    cat = star_catalog(spec.W, spec.H, spec.n_stars, g)
    R = add_noise(render(cat, spec.W, spec.H), 30.0, g)
    I = None
    if with_second_epoch:
        W, H = spec.W, spec.H
        def extra(x, y):
            return 0.6 + 0.3 * (x / max(W - 1, 1)) + 0.2 * (y / max(H - 1, 1))
        def fscale(x, y):
            return 1.02 - 0.04 * (y / max(H - 1, 1))
        I = add_noise(render(cat, W, H, extra_sigma=extra, flux_scale=fscale), 30.0, g)
    return R, I, cat


# ---------------------------------------------------------------- coefficient network inputs
CNN_IN = 64        # stamp side
CNN_CH = 32        # channels of every hidden layer
CNN_LAYERS = ((2, 2), (CNN_CH, 2), (CNN_CH, 2), (CNN_CH, 1))  # (input channels, stride) of the 4 convs


def cnn_param_shapes(n_out: int):
    """Parameter tensors of the coefficient network, in the flat order both the oracle
    and the CUDA library use: per conv layer w[Cout][Cin][3][3] then b[Cout], then the
    linear layer w[n_out][CNN_CH] and b[n_out]."""
    shapes = []
    for cin, _ in CNN_LAYERS:
        shapes.append((CNN_CH, cin, 3, 3))
        shapes.append((CNN_CH,))
    shapes.append((n_out, CNN_CH))
    shapes.append((n_out,))
    return shapes


def cnn_init_params(n_out: int, seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (float32 flat vector)."""
    g = rng(seed)
    out = []
    for shp in cnn_param_shapes(n_out):
        if len(shp) == 1:
            out.append(np.zeros(shp))
        else:
            fan_in = int(np.prod(shp[1:]))
            lim = math.sqrt(6.0 / fan_in)
            out.append(g.uniform(-lim, lim, shp))
    return np.concatenate([a.reshape(-1) for a in out]).astype(np.float32)
