"""Shared helpers for the GPU parity tests: seeded inputs and oracle references."""
import numpy as np

import oracle
import starfield

# Parity bar for the FP32 direct form and the split-precision (x3) tensor-core forms:
# max |D_gpu - D_oracle| <= 1e-5 * max |R (x) K| over the compared pixels.
TOL_FP32 = 1e-5


def star_pair(W, H, n_stars, seed, sky=1000.0):
    g = starfield.rng(seed)
    cat = starfield.star_catalog(W, H, n_stars, g)
    R = starfield.add_noise(starfield.render(cat, W, H, sky=sky), 30.0, g).astype(np.float32)
    I = starfield.add_noise(starfield.render(cat, W, H, sky=sky), 30.0, g).astype(np.float32)
    return R, I


def coeffs(N, degree, seed, **kw):
    return starfield.planted_coeffs(N, degree, starfield.rng(seed), **kw).astype(np.float32)


def oracle_conv(R, basis32, c32, degree, rows=None):
    """Oracle on exactly the float32 inputs the GPU sees (promoted to float64)."""
    return oracle.convolve(R.astype(np.float64), basis32.astype(np.float64), c32.astype(np.float64), degree, rows=rows)


def rel_err(gpu, ref, scale=None):
    scale = np.abs(ref).max() if scale is None else scale
    return float(np.abs(gpu.astype(np.float64) - ref).max() / scale)
