"""Parity of the direct form (FP32 FFMA on the CUDA cores) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _padded(a, pitch):
    t = torch.zeros((a.shape[0], pitch), dtype=torch.float32, device="cuda")
    t[:, : a.shape[1]] = _dev(a)
    return t[:, : a.shape[1]]


@pytest.mark.parametrize("W,H,L,d,pitch", [
    (256, 256, 11, 1, None),      # the 256x256 star-field case, full frame
    (300, 77, 19, 2, None),       # ragged tiles, TMA path (pitch multiple of 4)
    (47, 38, 7, 3, None),         # pitch 47: plain-load path
    (129, 9, 25, 0, 136),         # padded pitch, thin frame
    (1, 1, 5, 2, None),           # degenerate 1x1
    (5, 300, 31, 1, None),        # L > W
])
def test_direct_matches_oracle(W, H, L, d, pitch):
    R, I = star_pair(W, H, max(3, W * H // 300), 100 + W + H)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    N = B.shape[0]
    c = coeffs(N, d, 7)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    Rt = _dev(R) if pitch is None else _padded(R, pitch)
    out = svk.svk_convolve(Rt, B, _dev(c), d)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref) <= TOL_FP32
    D = svk.svk_difference(Rt, _dev(I), B, _dev(c), d)
    assert rel_err(D.cpu().numpy(), ref - I, scale=np.abs(ref).max()) <= TOL_FP32


@pytest.mark.parametrize("N", [1, 3, 8, 20, 49])
def test_direct_chunking_over_basis_count(N):
    W, H, L, d = 150, 40, 9, 2
    R, _ = star_pair(W, H, 30, 5)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)[:N].contiguous()
    c = coeffs(N, d, 8)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    out = svk.svk_convolve(_dev(R), B, _dev(c), d)
    assert rel_err(out.cpu().numpy(), ref) <= TOL_FP32


def test_direct_delta_basis_identity_and_dfb():
    W, H, L = 70, 50, 7
    R, _ = star_pair(W, H, 20, 9)
    B = svk.svk_build_basis(svk.SVK_BASIS_DELTA, L)
    N = L * L
    c = np.zeros((N, 1), np.float32)
    c[N // 2, 0] = 1.0
    out = svk.svk_convolve(_dev(R), B, _dev(c), 0)
    assert np.array_equal(out.cpu().numpy(), R)  # exact identity
    # the paper's workload: delta basis, second-order spatial polynomials
    c2 = coeffs(N, 2, 10)
    ref = oracle_conv(R, B.cpu().numpy(), c2, 2)
    out = svk.svk_convolve(_dev(R), B, _dev(c2), 2)
    assert rel_err(out.cpu().numpy(), ref) <= TOL_FP32


@pytest.mark.parametrize("kind,norm,L", [
    (svk.SVK_BASIS_GAUSS, svk.SVK_NORM_ALARD, 11), (svk.SVK_BASIS_GAUSS, svk.SVK_NORM_NONE, 19),
    (svk.SVK_BASIS_GAUSS, svk.SVK_NORM_ALARD, 31), (svk.SVK_BASIS_GAUSS, svk.SVK_NORM_ALARD, 63),
    (svk.SVK_BASIS_GAUSS, svk.SVK_NORM_NONE, 1), (svk.SVK_BASIS_DELTA, svk.SVK_NORM_ALARD, 5),
    (svk.SVK_BASIS_DELTA, svk.SVK_NORM_NONE, 3),
])
def test_build_basis_matches_oracle(kind, norm, L):
    B = svk.svk_build_basis(kind, L, normalize=norm).cpu().numpy()
    if kind == svk.SVK_BASIS_GAUSS:
        ref = oracle.gauss_basis(L, normalize=norm)
    else:
        ref = oracle.delta_basis(L, norm)
    scale = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)[:, None, None]
    assert np.abs(B - ref).max() <= 2 ** -23 * 4 * np.abs(ref).max() or np.all(np.abs(B - ref) <= 4e-7 * scale)
