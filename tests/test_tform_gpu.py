"""The T-factored form (sum_t m_t (R (x) K_t) - I, K_t = sum_k c[k][t] B_k) against the FP64
oracle of the per-pixel definition: the same result by linearity of Eq. 2 and 3."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP16X3, svk.SVK_PREC_FP32])
@pytest.mark.parametrize("W,H,L,d,kind", [
    (256, 256, 11, 1, svk.SVK_BASIS_GAUSS),
    (300, 177, 19, 2, svk.SVK_BASIS_GAUSS),   # many output rows per block, ragged
    (260, 90, 25, 3, svk.SVK_BASIS_GAUSS),
    (130, 61, 31, 0, svk.SVK_BASIS_GAUSS),
    (140, 50, 31, 3, svk.SVK_BASIS_GAUSS),   # the largest stamp table: T = 10 at L = 31
    (47, 38, 7, 2, svk.SVK_BASIS_DELTA),      # the paper's delta basis, L = 7
    (200, 70, 19, 2, svk.SVK_BASIS_DELTA),    # 361 delta stamps: beyond the basis form's N
    (1, 1, 5, 2, svk.SVK_BASIS_GAUSS),
])
def test_tform_matches_oracle(W, H, L, d, kind, prec):
    R, I = star_pair(W, H, max(3, W * H // 300), 600 + W + H)
    B = svk.svk_build_basis(kind, L)
    c = coeffs(B.shape[0], d, 13, const_sd=0.01, spatial_sd=0.005) if kind == svk.SVK_BASIS_DELTA else \
        coeffs(B.shape[0], d, 13)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    D = svk.svk_difference(_dev(R), _dev(I), B, _dev(c), d, method=svk.SVK_METHOD_TFORM, precision=prec)
    assert rel_err(D.cpu().numpy().astype(np.float64) + I, ref) <= TOL_FP32


@pytest.mark.parametrize("prec", [svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP32])
def test_tform_plain_convolution(prec):
    # svk_convolve (no I): R (x) K alone, through the same T-form kernels
    R, _ = star_pair(211, 97, 60, 777)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 15)
    c = coeffs(B.shape[0], 3, 5)
    ref = oracle_conv(R, B.cpu().numpy(), c, 3)
    out = svk.svk_convolve(_dev(R), B, _dev(c), 3, method=svk.SVK_METHOD_TFORM, precision=prec)
    assert rel_err(out.cpu().numpy().astype(np.float64), ref) <= TOL_FP32
